#!/usr/bin/env python
"""Benchmark: zone-cycles/s of the GR-MHD step on the 256^3 Fishbone-Moncrief
torus (MKS, r_out = 1000 M, a = 0.9375, gamma = 4/3, beta_0 = 100), mixed
precision (FP32 fluxes, FP64 conserved variables and inversion), with the
plain FP64 step timed beside it on the same GPU.

One JSON line on stdout (rank 0).  A "step" is one full RK2 step (both
stages, inversion, floors, fixups, boundaries and the CFL time step) of the
whole grid, replayed from a captured CUDA graph; inputs are resident in HBM.
The state (4.5 GB mixed, 7.7 GB FP64) is far larger than the 129 MB L2, so
no L2 flush is needed between steps.

Multi-GPU (torchrun, one rank per GPU): the one 256^3 torus split into N phi
slabs, rank r owning slab r (the slab layout of the paper's multi-GPU runs,
Section 3): the X3 ghost planes travel between neighbour ranks by NCCL
send/recv after each stage, the CFL minima by a MIN all-reduce (strong
scaling; the value is the whole grid's zone-cycles over the slowest rank's
time).  Independent replicas (one torus per rank, weak scaling) are a
secondary key.

--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HBM_BYTES_PER_ZONE_CYCLE = {"mixed": 344.0, "fp64": 472.0}
# algorithmic HBM bytes per zone of one stage update: the predictor reads P^n
# (8 x 4 B in the mixed path) and U^n (9 x 8 B) and writes P-hat; the corrector
# reads P-hat and U^n and writes U^{n+1} and P^{n+1} (their sum is the step's 344 B)
UPDATE_BYTES_PER_ZONE = {"pred": 136.0, "corr": 208.0}

# Algorithmic FP64 flops of the inversion of Section 2.3, from the oracle's
# operation counter (oracle/opcount.cpp: the oracle's own inversion compiled
# with a counting scalar; the figures are pinned by tests/test_oracle_opcount.py
# against a hand count): a Newton-only inversion costs C2P_FIXED_FLOPS (set-up
# 106, start 33, Newton constants 3, recovery 29) plus C2P_NEWTON_FLOPS per
# Newton step; the beta switch of the FP64 path (four-velocity and b^2 of the
# guess, gas pressure, beta test) adds C2P_BETA_FLOPS.  The stage update adds
# RK_FLOPS for U^n + dt_stage * rhs over the 9 conserved components.
C2P_FIXED_FLOPS = 171.0
C2P_NEWTON_FLOPS = 61.0
C2P_BETA_FLOPS = 120.0
RK_FLOPS = 18.0
# FP64 roofline from unit counts and clocks: 152 SMs x 2 FP64 FMA per clock
# x 2 flops x 2.07 GHz (the maximum SM clock); the FMA-chain probe is reported beside it
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes per zone of one k_update launch (dram__bytes_read.sum +
# dram__bytes_write.sum, ncu, one predictor launch of the 96^3 mixed torus;
# profiles/k_update_mixed_96cubed.md), valid while the kernel's sources hash to
# UPDATE_SOURCES_SHA (else the bench reports traffic null)
UPDATE_DRAM_BYTES_PER_ZONE = 257.4
UPDATE_SOURCES = ("stage_items.cuh", "con2prim.cuh", "fixes.cuh", "physics.cuh", "common.cuh", "step.cu")
UPDATE_SOURCES_SHA = "d27070c6ccddfed5"


def update_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in UPDATE_SOURCES:
        with open(os.path.join(ROOT, "paper_2205_02484_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    """HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=256, help="zones per direction (default 256)")
    ap.add_argument("--fp64-steps", type=int, default=0, help="FP64 steps (0: steps // 4, >= 3)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-mlp", action="store_true")
    ap.add_argument("--no-window", action="store_true")
    ap.add_argument("--no-slabs", action="store_true")
    ap.add_argument("--no-ppm", action="store_true")
    ap.add_argument("--slab-arm", action="store_true",
                    help="time the phi-slab decomposition (the multi-GPU arm) also at N = 1")
    return ap.parse_args()


def workload_config(n):
    return {"workload": f"3D Fishbone-Moncrief torus {n}^3 MKS, r_out=1000 M, a=0.9375, gamma=4/3, "
                        f"beta_min=100, 4% perturbation, mixed FP32-flux/FP64-inversion, PLM-MC+LLF+flux-CT",
            "grid": [n, n, n], "r_out": 1000.0, "spin": 0.9375, "gamma": 4.0 / 3.0, "beta0": 100.0,
            "r_in": 6.0, "r_max": 12.0, "precision": "mixed", "riemann": "LLF",
            "l2": "state (4.5 GB) exceeds L2 (129 MB); no flush needed",
            "graph": "one CUDA graph per RK2 step"}


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------- multi-rank

def max_over_ranks(x, dist=None, device=None):
    """Largest x over all ranks (the job's time is that of its slowest rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(zones_per_rank, steps, world, ms_max):
    """Whole-job zone-cycles/s: every rank advances its own grid."""
    return zones_per_rank * steps * world / (ms_max * 1e-3)


# -------------------------------------------------------------- ensemble

ENSEMBLE_SHAPES = [(64, 64, 1), (96, 64, 1), (128, 64, 32), (128, 96, 64), (192, 128, 64)]


SMALL_SHAPES = [(64, 64, 1), (96, 64, 1), (128, 64, 1), (64, 64, 4)]


def ensemble_specs(n=24, master_seed=2024, shapes=None):
    """Batched-ensemble workload: n tori with shapes drawn from 64x64x1 up to
    192x128x64, spin U[0, 0.98], gamma in {4/3, 13/9, 5/3}, beta_0 U[30, 300],
    perturbation seeds 100.. (one master seed)."""
    import numpy as np
    shapes = shapes or ENSEMBLE_SHAPES
    rng = np.random.Generator(np.random.PCG64(master_seed))
    out = []
    for m in range(n):
        shape = shapes[int(rng.integers(len(shapes)))]
        a = float(rng.uniform(0.0, 0.98))
        gam = [4.0 / 3.0, 13.0 / 9.0, 5.0 / 3.0][int(rng.integers(3))]
        b0 = float(rng.uniform(30.0, 300.0))
        out.append((shape, a, gam, b0, 100 + m))
    return out


def run_ensemble(G, torch, stream, device, steps=10, n=24, shapes=None, workload=None):
    """The batched ensemble against its members stepped one by one: the same
    contexts, all on one stream, each advancing by its own step graph in turn
    (the sequential loop); and a second set of contexts from the same draws,
    each on its own stream, whose step graphs the GPU overlaps (the
    concurrent loop).  All three start from the same initial states and are
    timed over the same number of steps after the same warm-up."""
    from paper_2205_02484_gb300 import tuning
    s = torch.cuda.Stream(device=device)

    def make(shared_stream):
        out = []
        for shape, a, gam, b0, seed in ensemble_specs(n=n, shapes=shapes):
            gp = G.default_grid(*shape, a=a, r_out=100.0, precision=G.MIXED, device=device)
            gp.stream = shared_stream.cuda_stream if shared_stream is not None else None
            c = G.init_grid(gp, G.default_phys(gam=gam))
            G.set_metric(c, a, G.KERR_MKS)
            G.init_torus(c, r_in=6.0, r_max=12.0, beta0=b0, pert_amp=0.04, seed=seed)
            out.append(c)
        return out

    def time_it(fn, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        fn(k)
        torch.cuda.synchronize()  # the concurrent loop's streams included
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def loop_of(ms):
        def loop(k):
            for _ in range(k):
                for c in ms:
                    G.step(c, 1)
        return loop

    members = make(s)
    zones = sum(c.nact for c in members)
    ens = G.ensemble_create(members)
    tiling, cached = tuning.tune_or_load(ens, torch.cuda.get_device_name(device), trial_steps=2)
    # the autotuner restored the initial states: every variant starts from them
    G.ensemble_step(ens, 2)
    ms_ens = time_it(lambda k: G.ensemble_step(ens, k), steps)
    G.ensemble_sync(ens)
    ens.close()
    for c in members:
        c.close()
    members = make(s)
    loop = loop_of(members)
    loop(2)
    ms_loop = time_it(loop, steps)
    for c in members:
        G.sync(c)
        c.close()
    members = make(None)
    loop = loop_of(members)
    loop(2)
    ms_conc = time_it(loop, steps)
    for c in members:
        G.sync(c)
        c.close()
    return {"workload": workload or ("24 FM tori, shapes 64x64x1..192x128x64, a U[0,0.98], gamma {4/3,13/9,5/3}, "
                                     "beta_0 U[30,300], r_out 100 M, mixed precision, one persistent launch per "
                                     "kernel class and one CUDA graph per ensemble step"),
            "members": n, "zones": zones, "steps": steps,
            "value": zones * steps / (ms_ens * 1e-3), "unit": "zone-cycles/s", "ms_per_step": ms_ens / steps,
            "loop_of_singles_value": zones * steps / (ms_loop * 1e-3),
            "loop_ms_per_step": ms_loop / steps, "speedup_vs_loop": ms_loop / ms_ens,
            "concurrent_streams_value": zones * steps / (ms_conc * 1e-3),
            "concurrent_ms_per_step": ms_conc / steps, "speedup_vs_concurrent_streams": ms_conc / ms_ens,
            "loop_note": "loop = the members' own step graphs one after another on one stream; "
                         "concurrent = the same on one stream per member (the GPU overlaps them)",
            "tiling": tiling, "tiling_from_cache": cached}


# ----------------------------------------------- theta slabs on one GPU

def run_theta_slabs(G, torch, device, n1=1024, n2=1024, steps=20, warmup=2, counts=(2, 4, 8)):
    """An n1 x n2 axisymmetric mixed torus split into R theta slabs on one GPU
    (decomp.ThetaRing: stage parts, X2 ghost rows through device buffers, the
    fixup loop of every stage on the device, one ring step captured in a CUDA
    graph and replayed), timed against the undecomposed graph step from the
    same state, with a bitwise comparison of the final states; the ring with
    the fixup loop run from the host (the failed-zone count read there once
    per stage and once per sweep, no graph) is timed too."""
    from paper_2205_02484_gb300.decomp import ThetaRing
    phys = G.default_phys(gam=13.0 / 9.0)
    gp = G.default_grid(n1, n2, 1, a=0.9375, r_out=1000.0, precision=G.MIXED, device=device)
    s = torch.cuda.Stream(device=device)
    gp.stream = s.cuda_stream
    full = G.init_grid(gp, phys)
    G.set_metric(full, 0.9375, G.KERR_MKS)
    G.init_torus(full, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=3)
    dev = f"cuda:{device}"
    P0 = torch.empty((8, n1, n2, 1), dtype=torch.float64, device=dev)
    U0 = torch.empty((9, n1, n2, 1), dtype=torch.float64, device=dev)
    _, _, t0, dt0 = G.get_state(full, P0, U0)

    def time_it(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    G.step(full, warmup)
    ms_full = time_it(lambda: G.step(full, steps))
    G.sync(full)
    Pf, Uf = torch.empty_like(P0), torch.empty_like(U0)
    G.get_state(full, Pf, Uf)
    nfix = G.diagnostics(full)["n_fixed"]
    full.close()
    out = {"workload": f"{n1}x{n2}x1 FM torus (axisymmetric), mixed precision, R theta slabs on one GPU",
           "steps": steps, "undecomposed_ms_per_step": ms_full / steps, "zones_fixed_undecomposed": nfix,
           "slabs": {}}
    for R in counts:
        ring = ThetaRing.create(gp, phys, R, 0.9375, stream=s)
        ring.set_state(P0, U0, t0, dt0)
        ring.step(warmup)
        ms = time_it(lambda: ring.step(steps))
        for e in ring.e:
            G.sync(e.ctx)
        parts = [_slab_state(G, torch, e, dev) for e in ring.e]
        Pr = torch.cat([p[0] for p in parts], dim=2)
        Ur = torch.cat([p[1] for p in parts], dim=2)
        del parts
        out["slabs"][str(R)] = {
            "ms_per_step": ms / steps, "vs_undecomposed": ms_full / ms,
            "bitwise_equal_to_undecomposed": bool(torch.equal(Pr, Pf) and torch.equal(Ur, Uf)),
            "ghost_bytes_per_slab_step": 4 * G.x2_row_bytes(ring.e[0].ctx, 0),
            "fixup_sweeps_last_step": list(ring.sweeps),
        }
        del Pr, Ur
        ring.close()
        host = ThetaRing.create(gp, phys, R, 0.9375, stream=s, device_fix=False)
        host.set_state(P0, U0, t0, dt0)
        host.step(warmup)
        out["slabs"][str(R)]["ms_per_step_host_loop"] = time_it(lambda: host.step(steps)) / steps
        host.close()
    return out


# ------------------------------------------------- phi slabs on one GPU

def run_slabs(G, torch, device, n, steps=10, warmup=2, counts=(2, 4, 8)):
    """The n^3 mixed torus split into R phi slabs on one GPU (decomp.SlabRing:
    stage-level launches, X3 ghost pack / unpack through device buffers, the
    per-direction dt minima folded on the device; one ring step captured in a
    CUDA graph and replayed, the host-launched form timed too), timed against the
    undecomposed graph step from the same state, with a bitwise comparison
    of the final states.  A slab's time per step approximates one rank's
    compute in an R-GPU run; ghost_bytes_per_slab_step is what that rank would
    send per step (2 stages x 2 sides x NG = 3 planes of 8 primitives)."""
    from paper_2205_02484_gb300.decomp import SlabRing
    phys = G.default_phys(gam=4.0 / 3.0)
    gp = G.default_grid(n, n, n, a=0.9375, r_out=1000.0, precision=G.MIXED, device=device)
    s = torch.cuda.Stream(device=device)
    gp.stream = s.cuda_stream
    full = G.init_grid(gp, phys)
    G.set_metric(full, 0.9375, G.KERR_MKS)
    G.init_torus(full, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=3)
    dev = f"cuda:{device}"
    P0 = torch.empty((8, n, n, n), dtype=torch.float64, device=dev)
    U0 = torch.empty((9, n, n, n), dtype=torch.float64, device=dev)
    _, _, t0, dt0 = G.get_state(full, P0, U0)

    def time_it(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    G.step(full, warmup)
    ms_full = time_it(lambda: G.step(full, steps))
    G.sync(full)
    Pf = torch.empty_like(P0)
    Uf = torch.empty_like(U0)
    G.get_state(full, Pf, Uf)
    full.close()
    out = {"workload": f"{n}^3 FM torus (the headline state), mixed precision, R phi slabs on one GPU",
           "steps": steps, "undecomposed_ms_per_step": ms_full / steps, "slabs": {}}
    for R in counts:
        ring = SlabRing.create(gp, phys, R, 0.9375, stream=s)
        ring.set_state(P0, U0, t0, dt0)
        ring.step(warmup)
        ms = time_it(lambda: ring.step(steps))
        for e in ring.e:
            G.sync(e.ctx)
        parts = [_slab_state(G, torch, e, dev) for e in ring.e]
        Pr = torch.cat([p[0] for p in parts], dim=3)
        Ur = torch.cat([p[1] for p in parts], dim=3)
        del parts
        out["slabs"][str(R)] = {
            "ms_per_step": ms / steps, "vs_undecomposed": ms_full / ms,
            "bitwise_equal_to_undecomposed": bool(torch.equal(Pr, Pf) and torch.equal(Ur, Uf)),
            "ghost_bytes_per_slab_step": 4 * G.x3_plane_bytes(ring.e[0].ctx),
            # per slab: 2 stages x 10 kernels, dt minima, finish; 2 exchanges x 4
            "launches_per_step": R * (2 * 10 + 2 + 2 * 4),
        }
        del Pr, Ur
        out["slabs"][str(R)]["ms_per_step_host_launches"] = time_it(lambda: ring.step(steps, graph=False)) / steps
        ring.close()
    return out


def _slab_state(G, torch, e, dev):
    n1, n2, n3 = e.ctx.shape
    P = torch.empty((8, n1, n2, n3), dtype=torch.float64, device=dev)
    U = torch.empty((9, n1, n2, n3), dtype=torch.float64, device=dev)
    G.get_state(e.ctx, P, U)
    return P, U


# ---------------------------------------------- stand-alone inversion

# FP64 flops per inversion of k_con2prim on these states (ncu count of DFMA x 2
# + DMUL + DADD, 1e6 inversions from a guess within 1e-4): see the profile
# summary of the kernel


def run_con2prim(G, torch, stream, device, n=1_000_000, rel=1e-4):
    """Batched inversions (Section 2.3, FP64 path with its confirmation
    step) of n seeded states from the learned-start sample distribution at
    the 256x192 grid's metric, each started from its exact primitives
    perturbed by up to `rel` (what the previous stage hands the step)."""
    gp = G.default_grid(256, 192, 1, a=0.9375, r_out=1000.0, precision=G.FP64, device=device)
    gp.stream = stream.cuda_stream
    ctx = G.init_grid(gp, G.default_phys(gam=4.0 / 3.0))
    G.set_metric(ctx, 0.9375, G.KERR_MKS)
    P, loc, U, f, y = G.mlp_samples(ctx, 11, 0, n, device=True)
    gen = torch.Generator(device=P.device).manual_seed(5)
    g0 = P.clone()
    g0[:5] *= 1.0 + rel * (2.0 * torch.rand((5, n), generator=gen, device=P.device, dtype=torch.float64) - 1.0)
    flags = torch.zeros(n, dtype=torch.int32, device=P.device)
    iters = torch.zeros(n, dtype=torch.int32, device=P.device)
    G.con2prim(ctx, U, loc, g0.clone(), flags, iters)
    best = None
    for _ in range(3):
        work = g0.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.con2prim(ctx, U, loc, work, flags, iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    fl = flags.cpu().numpy()
    it = iters.cpu().numpy()
    # the Newton branch alone, the inversions the torus step runs: the draws
    # that took it above, inverted again as one batch from the same guesses
    idx = torch.nonzero(flags == 0).squeeze(1)
    m = int(idx.numel())
    Un, ln, gn = U[:, idx].contiguous(), loc[idx].contiguous(), g0[:, idx].contiguous()
    fl2 = torch.zeros(m, dtype=torch.int32, device=P.device)
    it2 = torch.zeros(m, dtype=torch.int32, device=P.device)
    G.con2prim(ctx, Un, ln, gn.clone(), fl2, it2)
    best2 = None
    for _ in range(3):
        work = gn.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.con2prim(ctx, Un, ln, work, fl2, it2)
        e1.record(stream)
        torch.cuda.synchronize()
        ms2 = e0.elapsed_time(e1)
        best2 = ms2 if best2 is None else min(best2, ms2)
    f2 = fl2.cpu().numpy()
    i2 = it2.cpu().numpy()
    ctx.close()
    out = {"workload": f"{n} inversions (FP64 path), states of the seeded sample distribution at the 256x192 "
                       f"grid's metric, guess = exact primitives x (1 + {rel} U[-1,1])",
           "ms": best, "inversions_per_s": n / (best * 1e-3),
           "newton_iters_mean": float(it[fl == 0].mean()), "frac_newton": float((fl == 0).mean()),
           "frac_entropy_beta": float((fl == 3).mean()), "frac_fail": float(((fl & 8) != 0).mean())}
    # algorithmic flops of the Newton inversions (oracle op counter); the
    # entropy-branch zones are left out of the numerator (a lower bound)
    nr = fl == 0
    flops = float(((C2P_FIXED_FLOPS + C2P_BETA_FLOPS) + C2P_NEWTON_FLOPS * it[nr]).sum())
    tf = flops / (best * 1e-3) / 1e12
    out.update({"fp64_flops_newton_inversions": flops,
                "flops_per_newton_inversion": flops / max(int(nr.sum()), 1),
                "tflops_fp64_algorithmic": tf, "frac_of_fp64_peak": tf / FP64_PEAK_TFLOPS,
                "fp64_peak_tflops": FP64_PEAK_TFLOPS,
                "flops_source": "oracle operation counter (oracle/opcount.cpp), Newton inversions only"})
    flops2 = float(((C2P_FIXED_FLOPS + C2P_BETA_FLOPS) + C2P_NEWTON_FLOPS * i2[f2 == 0]).sum())
    tf2 = flops2 / (best2 * 1e-3) / 1e12
    out["newton_branch"] = {
        "workload": f"the {m} draws above that Newton inverts, as one batch from the same guesses",
        "ms": best2, "inversions_per_s": m / (best2 * 1e-3), "all_newton": bool((f2 == 0).all()),
        "newton_iters_mean": float(i2[f2 == 0].mean()) if m else 0.0,
        "tflops_fp64_algorithmic": tf2, "frac_of_fp64_peak": tf2 / FP64_PEAK_TFLOPS}
    return out


# ------------------------------------------- mixed vs FP64 short window

def run_window(G, torch, stream, device, n=128, steps=200, every=10, gam=4.0 / 3.0, beta0=100.0, pert=0.02, seed=2):
    """The first `steps` steps of the n^3 torus (gamma, beta_0, perturbation,
    seed as given) from the same initial state in FP64 and in mixed
    precision: horizon Mdot and phi_B every `every` steps, and the per-field
    deviation of the final state (the FP64 GPU step is held to the FP64
    oracle at 1e-10 per step by the parity tests)."""
    import numpy as np
    series, finals = {}, {}
    for name, prec in (("fp64", G.FP64), ("mixed", G.MIXED)):
        gp = G.default_grid(n, n, n, a=0.9375, r_out=1000.0, precision=prec, device=device)
        gp.stream = stream.cuda_stream
        c = G.init_grid(gp, G.default_phys(gam=gam))
        G.set_metric(c, 0.9375, G.KERR_MKS)
        G.init_torus(c, r_in=6.0, r_max=12.0, beta0=beta0, pert_amp=pert, seed=seed)
        if name == "fp64":
            P0, U0, t0, dt0 = G.get_state(c)
        else:
            G.set_state(c, P0, U0, t0, dt0)
        rows = []
        for k in range(steps // every):
            G.step(c, every)
            d = G.diagnostics(c)
            rows.append((d["t"], d["mdot"], d["phib"]))
        series[name] = np.array(rows)
        finals[name] = G.get_state(c)
        c.close()
    a, b = series["fp64"], series["mixed"]
    Pa, Ua = finals["fp64"][:2]
    Pb, Ub = finals["mixed"][:2]
    body = Pa[0] > 1e-3 * Pa[0].max()   # zones of the torus body (off the floored atmosphere)

    def field_dev(x, y, positive):
        out = []
        for f in range(x.shape[0]):
            if f in positive:
                out.append(float(np.max(np.abs(y[f] - x[f]) / np.abs(x[f]))))
            else:
                out.append(float(np.max(np.abs(y[f] - x[f])) / max(np.max(np.abs(x[f])), 1e-300)))
        return out
    return {"workload": f"{n}^3 FM torus, gamma {gam:.4g}, beta_0 {beta0:g}, {100 * pert:g}% perturbation, seed "
                        f"{seed}; first {steps} steps from the same initial state, FP64 vs mixed",
            "t_end": float(a[-1, 0]),
            # normwise over the series
            "mdot_max_rel_dev": float(np.max(np.abs(b[:, 1] - a[:, 1])) / max(np.max(np.abs(a[:, 1])), 1e-300)),
            "phib_max_rel_dev": (float(np.max(np.abs(b[:, 2] - a[:, 2])) / np.max(np.abs(a[:, 2])))
                                 if np.max(np.abs(a[:, 2])) > 1e-30 else None),
            "phib_note": ("the loop field lies inside the torus: phi_B at the horizon is zero in this window "
                          "(the split-monopole test of the mixed path covers phi_B)"
                          if np.max(np.abs(a[:, 2])) <= 1e-30 else None),
            "mdot_fp64_last": float(a[-1, 1]), "phib_fp64_last": float(a[-1, 2]),
            "prim_dev_final_torus_body": field_dev(Pa[:, body], Pb[:, body], (0, 1)),
            "prim_dev_final": field_dev(Pa, Pb, (0, 1)),
            "cons_dev_final": field_dev(Ua, Ub, (0, 1, 8)),
            "metric_note": "pointwise relative for rho, u (U_rho, U_E, U_S), max-norm relative for the others"}


def run_variants(G, torch, stream, device, n=256, steps=20, warmup=3):
    """The 256^3 mixed step at each (gamma, beta_0) of {4/3, 5/3} x {100, 30}:
    zone-cycles/s, Newton steps per zone and fallback counts."""
    out = []
    for gam in (4.0 / 3.0, 5.0 / 3.0):
        for b0 in (100.0, 30.0):
            gp = G.default_grid(n, n, n, a=0.9375, r_out=1000.0, precision=G.MIXED, device=device)
            gp.stream = stream.cuda_stream
            c = G.init_grid(gp, G.default_phys(gam=gam))
            G.set_metric(c, 0.9375, G.KERR_MKS)
            G.init_torus(c, r_in=6.0, r_max=12.0, beta0=b0, pert_amp=0.04, seed=3)
            G.step(c, warmup)
            G.sync(c)
            d0 = G.diagnostics(c)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            G.step(c, steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            d1 = G.diagnostics(c)
            nr = max(d1["n_nr"] - d0["n_nr"], 1)
            out.append({"gamma": gam, "beta0": b0, "value": n ** 3 * steps / (ms * 1e-3), "unit": "zone-cycles/s",
                        "ms_per_step": ms / steps,
                        "newton_steps_per_zone": (d1["nr_iters"] - d0["nr_iters"]) / nr,
                        "fallbacks": {k: d1[k] - d0[k] for k in ("n_brent", "n_entropy", "n_entropy_beta", "n_fail",
                                                                 "n_ceil", "n_gcap")}})
            c.close()
    return {"workload": f"{n}^3 FM torus, r_out 1000 M, a 0.9375, 4% perturbation, mixed precision; {steps} steps "
                        f"after {warmup}", "runs": out}


# ------------------------------------------------------- learned Newton start

# FP32 flops per training sample of the 5-64-64-1 network: forward
# 2 (5*64 + 64*64 + 64); backward dh1 = W2^T dh2 (2*64*64), dW2 (2*64*64),
# dW1 (2*64*5), dW3, db (3*2*64)
MLP_TRAIN_FLOPS = 2 * (5 * 64 + 64 * 64 + 64) + 2 * 64 * 64 * 2 + 2 * 64 * 5 + 3 * 2 * 64


def counters(G, ctx):
    d = G.diagnostics(ctx)
    return {k: d[k] for k in ("nr_iters", "n_nr", "n_brent", "n_entropy", "n_entropy_beta", "n_fail", "n_fixed",
                              "n_learned")}


def run_mlp(G, torch, stream, device, fp32_peak, n_samples=10_000_000, epochs=4, steps=10):
    """Train the learned Newton start on the GPU, compare inversions from a
    poor start with and without it, and time the 256x192x192 mixed step with
    the plain and the learned start."""
    gp = G.default_grid(256, 192, 192, a=0.9375, r_out=1000.0, precision=G.MIXED, device=device)
    gp.stream = stream.cuda_stream
    ctx = G.init_grid(gp, G.default_phys(gam=4.0 / 3.0))
    G.set_metric(ctx, 0.9375, G.KERR_MKS)
    rep = G.mlp_train(ctx, n_samples=n_samples, n_val=100_000, seed=7, init_seed=1, epochs=epochs, batch=4096,
                      lr=2e-3, lr_min=2e-5, weight_decay=1e-4)
    train = dict(rep)
    train["tflops_fp32"] = rep["samples_per_s"] * MLP_TRAIN_FLOPS / 1e12
    train["frac_of_fp32_probe"] = train["tflops_fp32"] / fp32_peak if fp32_peak else None
    train["flops_per_sample"] = MLP_TRAIN_FLOPS

    def ev_time(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # held-out states; the poor start knows rho, u and B but not the flow (no velocity)
    n = 1_000_000
    P, loc, U, f, y = G.mlp_samples(ctx, 7, 50_000_000, n, device=True)
    inv = {}
    for name, learned in (("plain_static_start", 0), ("learned_start", 1), ("learned_rescue", 2)):
        g0 = P.clone()
        g0[2:5] = 0.0
        flags = torch.zeros(n, dtype=torch.int32, device=P.device)
        iters = torch.zeros(n, dtype=torch.int32, device=P.device)
        G.con2prim(ctx, U, loc, g0.clone(), flags, iters, use_learned_guess=learned)   # warm
        ms = ev_time(lambda: G.con2prim(ctx, U, loc, g0, flags, iters, use_learned_guess=learned))
        fl = flags.cpu().numpy()
        it = iters.cpu().numpy()
        nr = fl == 0
        nr = (fl & 7) == 0
        nr &= (fl & 8) == 0
        inv[name] = {"ms": ms, "inversions_per_s": n / (ms * 1e-3), "newton_iters_mean": float(it[nr].mean()),
                     "frac_newton": float(nr.mean()), "frac_brent": float((fl == 1).mean()),
                     "frac_learned_rescue": float(((fl & 64) != 0).mean()),
                     "frac_entropy": float((fl == 2).mean()), "frac_entropy_beta": float((fl == 3).mean()),
                     "frac_fail": float(((fl & 8) != 0).mean())}
    # the zone class Newton serves: the draws the plain order inverts by Newton
    # (not the beta < 1e-2 entropy ones), compacted, the same two starts
    g0 = P.clone()
    g0[2:5] = 0.0
    flags = torch.zeros(n, dtype=torch.int32, device=P.device)
    iters = torch.zeros(n, dtype=torch.int32, device=P.device)
    G.con2prim(ctx, U, loc, g0.clone(), flags, iters)
    sel = torch.nonzero(flags == 0).flatten()
    Us, ls, gs = U[:, sel].contiguous(), loc[sel].contiguous(), g0[:, sel].contiguous()
    m = int(sel.numel())
    newton_zones = {"zones": m}
    for name, learned in (("plain_static_start", 0), ("learned_start", 1)):
        fs = torch.zeros(m, dtype=torch.int32, device=P.device)
        its = torch.zeros(m, dtype=torch.int32, device=P.device)
        G.con2prim(ctx, Us, ls, gs.clone(), fs, its, use_learned_guess=learned)   # warm
        ms = ev_time(lambda: G.con2prim(ctx, Us, ls, gs.clone(), fs, its, use_learned_guess=learned))
        it = its.cpu().numpy()
        newton_zones[name] = {"ms": ms, "inversions_per_s": m / (ms * 1e-3), "newton_iters_mean": float(it.mean()),
                              "frac_newton": float(((fs & 15) == 0).float().mean().item())}
    newton_zones["note"] = ("the inversion with the learned start first evaluates the network on the tensor cores "
                            "(warp-level BF16 MMA, FP32 accumulation); the clone of the start is inside both times")
    inv["newton_zone_class"] = newton_zones
    g0 = P.clone()
    flags = torch.zeros(n, dtype=torch.int32, device=P.device)
    iters = torch.zeros(n, dtype=torch.int32, device=P.device)
    G.con2prim(ctx, U, loc, g0, flags, iters)
    fl, it = flags.cpu().numpy(), iters.cpu().numpy()
    inv["exact_prims_start"] = {"newton_iters_mean": float(it[fl == 0].mean()), "frac_newton": float((fl == 0).mean())}

    # the 256x192x192 step: plain order (previous-stage primitives, extrapolated)
    # vs the learned rescue before Brent
    G.init_torus(ctx, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.02, seed=2)
    zones = ctx.nact
    step = {}
    for name, learned in (("plain_start", False), ("learned_rescue", True)):
        G.set_learned_guess(ctx, learned)
        G.step(ctx, 2)
        c0 = counters(G, ctx)
        ms = ev_time(lambda: G.step(ctx, steps))
        c1 = counters(G, ctx)
        d = {k: c1[k] - c0[k] for k in c0}
        inversions = 2 * zones * steps
        step[name] = {"value": zones * steps / (ms * 1e-3), "unit": "zone-cycles/s", "ms_per_step": ms / steps,
                      "newton_iters_per_newton_zone": d["nr_iters"] / max(d["n_nr"], 1),
                      "fallback_per_inversion": (d["n_brent"] + d["n_entropy"]) / inversions,
                      "entropy_beta_per_inversion": d["n_entropy_beta"] / inversions,
                      "fail_per_inversion": d["n_fail"] / inversions,
                      "learned_rescue_per_inversion": d["n_learned"] / inversions}
    G.set_learned_guess(ctx, False)
    # the zone class the rescue serves: the first step after a restart whose
    # primitives know rho, u and B but not the flow (velocities zero), with
    # Newton capped at 8 steps; without the network the zones that need more
    # Newton steps from that start take the 1D Brent solve
    th, nm = G.mlp_get(ctx)
    gp8 = G.default_grid(256, 192, 192, a=0.9375, r_out=1000.0, precision=G.MIXED, device=device)
    gp8.stream = stream.cuda_stream
    c8 = G.init_grid(gp8, G.default_phys(gam=4.0 / 3.0, nr_maxit=8))
    G.set_metric(c8, 0.9375, G.KERR_MKS)
    G.mlp_load(c8, th, nm)
    G.init_torus(c8, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.02, seed=2)
    G.step(c8, 5)
    Pd = torch.empty((8,) + c8.shape, dtype=torch.float64, device=f"cuda:{device}")
    Ud = torch.empty((9,) + c8.shape, dtype=torch.float64, device=f"cuda:{device}")
    _, _, t8, dt8 = G.get_state(c8, Pd, Ud)
    Pd[2:5] = 0.0
    restart = {}
    for name, learned in (("plain_start", False), ("learned_rescue", True)):
        G.set_learned_guess(c8, learned)
        G.set_state(c8, Pd, Ud, t8, dt8)
        G.step(c8, 1)   # the graph is captured on the first call: time the second restart
        G.set_state(c8, Pd, Ud, t8, dt8)
        c0 = counters(G, c8)
        ms = ev_time(lambda: G.step(c8, 1))
        c1 = counters(G, c8)
        d = {k: c1[k] - c0[k] for k in c0}
        restart[name] = {"ms_first_step": ms, "brent": d["n_brent"], "learned_rescue": d["n_learned"],
                         "entropy": d["n_entropy"], "fail": d["n_fail"],
                         "newton_iters_per_zone_stage": d["nr_iters"] / (2.0 * zones)}
    G.set_learned_guess(c8, False)
    c8.close()
    del Pd, Ud
    ctx.close()
    return {"workload": "learned Newton start: 5-64-64-1 MLP, BF16 weights, FP32 accumulate; trained on the GPU "
                        f"on {n_samples} seeded samples x {epochs} epochs (log-uniform rho in [1e-6,1], u/rho in "
                        "[1e-4,10], Gamma in [1,50], b^2/rho in [1e-3,100]) at the 256x192x192 MKS grid's metric; "
                        "step: 256x192x192 FM torus, mixed precision",
            "train": train, "inversion_1e6_heldout": inv, "step_256x192x192": step,
            "restart_no_velocity_newton_cap_8": restart}


# ------------------------------------------------------------ CPU oracle

def oracle_sample_run(n, n3s, steps, warmup):
    """The FP64 CPU oracle, as it stands, on an n x n x n3s slab of the
    workload (same r, theta grid; n3s phi zones).  Returns (zone-cycles/s,
    seconds, description)."""
    import oracle
    p = oracle.default_params(n1=n, n2=n, n3=n3s, gam=4.0 / 3.0, r_out=1000.0, a=0.9375)
    og = oracle.Grid(p)
    og.init_torus(r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=3)
    if warmup:
        og.step(warmup)
    t0 = time.perf_counter()
    og.step(steps)
    dt = time.perf_counter() - t0
    zc = n * n * n3s * steps / dt
    desc = (f"{n}x{n}x{n3s} phi-slab of the {n}^3 torus (same r, theta grid), {steps} RK2 steps "
            f"after {warmup} warm-up, single-threaded plain C -O2")
    return zc, dt, desc


def oracle_timed(n1, n2, n3, steps, gam, r_out, seed):
    """Single-threaded oracle zone-cycles/s of an n1 x n2 x n3 torus (seeded
    perturbation 0.04, beta_0 100) over `steps` RK2 steps."""
    import oracle
    og = oracle.Grid(oracle.default_params(n1=n1, n2=n2, n3=n3, gam=gam, r_out=r_out, a=0.9375))
    og.init_torus(r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=seed)
    t0 = time.perf_counter()
    og.step(steps)
    return n1 * n2 * n3 * steps / (time.perf_counter() - t0)


def _oracle_core_worker(job):
    """one host core's share for oracle_all_cores: its own n x n x n3s slab
    torus, `steps` timed steps"""
    n, n3s, steps, seed = job
    import oracle
    p = oracle.default_params(n1=n, n2=n, n3=n3s, gam=4.0 / 3.0, r_out=1000.0, a=0.9375)
    og = oracle.Grid(p)
    og.init_torus(r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=seed)
    t0 = time.perf_counter()
    og.step(steps)
    return time.perf_counter() - t0


def oracle_all_cores(n, n3s, steps):
    """The same oracle on every host core at once: one n x n x n3s slab per
    core in its own process (spawned), as a phi-slab decomposition of an
    n x n x (cores n3s) grid would run it without the ghost exchange.  Returns
    (zone-cycles/s of all cores, cores, description)."""
    import multiprocessing as mp
    cores = max(1, min(os.cpu_count() or 1, 144))
    with mp.get_context("spawn").Pool(cores) as pool:
        times = pool.map(_oracle_core_worker, [(n, n3s, steps, 3 + c) for c in range(cores)])
    zc = cores * n * n * n3s * steps / max(times)
    from oracle import NG
    desc = (f"{cores} processes, each a {n}x{n}x{n3s} phi-slab of the {n}^3 torus, {steps} RK2 steps timed "
            f"per process; the job time is the slowest process's (the ghost exchange of a decomposed run, "
            f"{2 * NG * 8 * (n + 2 * NG) ** 2 * 8 / 1e6:.1f} MB per slab and stage, left out)")
    return zc, cores, desc


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.n
    # per-step work bounded so that warmup + steps finish in about a minute
    n3s = 1 if args.steps + args.warmup > 10 else 2
    zc, dt, desc = oracle_sample_run(n, n3s, args.steps, args.warmup)
    line = {"impl": "reference", "metric": "zone-cycles/s at 256^3 (FP64 vs mixed, same GB300); % of HBM roofline",
            "value": zc, "unit": "zone-cycles/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(n),
            "cpu_baseline": {"value": zc, "unit": "zone-cycles/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": zc, "unit": "zone-cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- GPU arm

def run_ppm(G, torch, stream, device, n=256, steps=10, warmup=3):
    """The headline workload with PPM faces (GRMHD_PPM) instead of PLM: the
    step time and the share of its face sweeps (CUDA events between kernel
    groups)."""
    gp = G.default_grid(n, n, n, a=0.9375, r_out=1000.0, precision=G.MIXED, device=device, recon=G.PPM)
    gp.stream = stream.cuda_stream
    ctx = G.init_grid(gp, G.default_phys(gam=4.0 / 3.0))
    G.set_metric(ctx, 0.9375, G.KERR_MKS)
    G.init_torus(ctx, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=3)
    G.step(ctx, warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    G.step(ctx, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof = G.step_profiled(ctx, 2)
    flux = sum(prof[f"flux_x{d}_{s}"] for d in (1, 2, 3) for s in ("pred", "corr")) / 2.0
    d = G.diagnostics(ctx)
    ctx.close()
    return {"workload": f"the {n}^3 torus of the headline with PPM faces (six-zone stencil; X1 / X2 columns, X3 row warps)",
            "value": n ** 3 / (ms * 1e-3), "unit": "zone-cycles/s", "ms_per_step": ms,
            "face_sweeps_ms_per_step": flux, "n_fail": d["n_fail"], "divb_max": d["divb_max"]}


def run_decomposed(G, torch, dist, world, rank, local, n, steps, warmup, barrier):
    """The phi-slab decomposition of one n^3 torus over the ranks: the
    headline of a multi-GPU run.  Every rank builds the whole initial torus
    (seed 3), keeps its slab, frees the rest, and steps its slab; the
    exchanges run on the slab's stream."""
    from paper_2205_02484_gb300 import decomp as D
    base = G.default_grid(n, n, n, a=0.9375, r_out=1000.0, precision=G.MIXED, device=local)
    phys = G.default_phys(gam=4.0 / 3.0)
    sstream = torch.cuda.Stream(device=local)
    eng = D.CtxSlab.create(D.slab_grid(base, world), phys, 0.9375, sstream)
    slab = D.SlabRank(eng)
    full_g = G.GridParams.from_buffer_copy(base)
    full_g.stream = sstream.cuda_stream
    full = G.init_grid(full_g, phys)
    G.set_metric(full, 0.9375, G.KERR_MKS)
    G.init_torus(full, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=3)
    dev = f"cuda:{local}"
    P = torch.empty((8, n, n, n), dtype=torch.float64, device=dev)
    U = torch.empty((9, n, n, n), dtype=torch.float64, device=dev)
    _, _, t0, dt0 = G.get_state(full, P, U)
    full.close()
    slab.set_state(P, U, t0, dt0)
    del P, U
    torch.cuda.empty_cache()
    slab.step(warmup)
    torch.cuda.synchronize()
    clk = ClockSampler(local if world > 1 else None)
    barrier()
    clk.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(sstream)
    slab.step(steps)
    e1.record(sstream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    clocks = clk.stop()
    diag = slab.diagnostics()
    zones = n * n * n
    # end to end: each rank copies its slab's state in from pinned host
    # buffers, steps, and copies it back, every step
    n3 = n // world
    Ph = torch.empty((8, n, n, n3), dtype=torch.float64, pin_memory=True).numpy()
    Uh = torch.empty((9, n, n, n3), dtype=torch.float64, pin_memory=True).numpy()
    _, _, t, dt = G.get_state(eng.ctx, Ph, Uh)
    ne = 3
    barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(ne):
        G.set_state(eng.ctx, Ph, Uh, t, dt)
        slab.exchange(0)
        slab.step(1)
        _, _, t, dt = G.get_state(eng.ctx, Ph, Uh)
    torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - w0, dist, "cuda")
    e2e = {"value": zones * ne / el, "unit": "zone-cycles/s",
           "h2d_bytes_per_step": int(17 * 8 * zones), "d2h_bytes_per_step": int(17 * 8 * zones), "steps": ne,
           "path": "per rank: grmhd_set_state(host slab) + ghost exchange + the slab step + grmhd_get_state(host "
                   "slab), pinned buffers"}
    eng.close()
    return {"value": zones * steps / (ms * 1e-3), "ms_per_step": ms / steps, "clocks": clocks, "e2e": e2e,
            "diag": {k: diag[k] for k in ("t", "dt", "mdot", "divb_max", "n_fail", "nr_iters", "n_steps")},
            "launches_per_step": 2 * 10 + 2 + 2 * 4}  # stages of 10 kernels, dt minima and finish, 2 exchanges


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2205_02484_gb300 import grmhd as G
    G.load(build_if_missing=True)
    n = args.n
    stream = torch.cuda.current_stream()

    def make_ctx(precision):
        gp = G.default_grid(n, n, n, a=0.9375, r_out=1000.0, precision=precision, device=local)
        gp.stream = stream.cuda_stream
        ctx = G.init_grid(gp, G.default_phys(gam=4.0 / 3.0))
        G.set_metric(ctx, 0.9375, G.KERR_MKS)
        G.init_torus(ctx, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=3 + rank)
        return ctx

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(ctx, steps, warmup, sample_clocks):
        G.step(ctx, warmup)
        G.sync(ctx)
        clk = ClockSampler(local if world > 1 else None) if sample_clocks else None
        barrier()
        torch.cuda.synchronize()
        if clk:
            clk.start()
            time.sleep(0.3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.step(ctx, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        clocks = clk.stop() if clk else None
        G.sync(ctx)
        ms = max_over_ranks(ms, dist, "cuda")
        return ms, clocks

    zones = n * n * n
    if world > 1 or args.slab_arm:
        if dist is None:  # --slab-arm on one GPU: a one-rank group
            import socket
            import torch.distributed as dist
            sk = socket.socket()
            sk.bind(("127.0.0.1", 0))
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", str(sk.getsockname()[1]))
            sk.close()
            dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", local))
        dec = run_decomposed(G, torch, dist, world, rank, local, n, args.steps, args.warmup, lambda: dist.barrier())
        # secondary: independent replicas, one torus per rank (weak scaling)
        rctx = make_ctx(G.MIXED)
        rms, _ = timed(rctx, 10, min(args.warmup, 3), False)
        rctx.close()
        replicas = {"value": aggregate_value(zones, 10, world, rms), "unit": "zone-cycles/s", "steps": 10,
                    "ms_per_step": rms / 10, "scaling": "weak",
                    "path": "one 256^3 torus per rank (seed 3 + rank), no communication"}
        if rank == 0:
            line = {
                "metric": "zone-cycles/s at 256^3 (FP64 vs mixed, same GB300); % of HBM roofline",
                "value": dec["value"], "unit": "zone-cycles/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dec["ms_per_step"], "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32 fluxes + f64 U/inversion",
                "data": "synthetic",
                "config": dict(workload_config(n), parallelism=f"phi slabs x{world} (one 256^3 torus)",
                               graph="none: host-driven stages, X3 ghost planes by NCCL send/recv, dt by a MIN "
                                     "all-reduce"),
                "hbm_roofline": {"bytes_per_zone_cycle": HBM_BYTES_PER_ZONE_CYCLE["mixed"],
                                 "achieved_gbs": HBM_BYTES_PER_ZONE_CYCLE["mixed"] * dec["value"] / 1e9},
                "clocks": dec["clocks"], "e2e": dec["e2e"], "gpu_launches": dec["launches_per_step"] * args.steps,
                "replicas": replicas, "diagnostics_after_bench": dec["diag"],
            }
            print(json.dumps(line), flush=True)
        dist.destroy_process_group()
        return
    # ---- headline: mixed precision
    ctx = make_ctx(G.MIXED)
    ms, clocks = timed(ctx, args.steps, args.warmup, True)
    value = aggregate_value(zones, args.steps, world, ms)
    ms_step = ms / args.steps
    # the same step by windows: 5 windows of 20 steps, their median (the
    # headline above is one window of exactly `steps` steps)
    windows = None
    d_w0 = G.diagnostics(ctx)
    if world == 1:
        wms = []
        for _ in range(5):
            w0 = torch.cuda.Event(enable_timing=True)
            w1 = torch.cuda.Event(enable_timing=True)
            w0.record(stream)
            G.step(ctx, 20)
            w1.record(stream)
            torch.cuda.synchronize()
            wms.append(w0.elapsed_time(w1) / 20)
        med = statistics.median(wms)
        windows = {"windows": 5, "steps_per_window": 20, "ms_per_step": wms,
                   "median_ms_per_step": med, "median_value": zones / (med * 1e-3)}
        G.sync(ctx)
    diag = G.diagnostics(ctx)
    # barycentric radius of Eq. 43 (r_bar_max = 80 M), timed on its own
    G.barycentric_radius(ctx, 80.0)
    b0 = time.perf_counter()
    for _ in range(5):
        bary = G.barycentric_radius(ctx, 80.0)
    bary_ms = (time.perf_counter() - b0) * 1e3 / 5
    # horizon diagnostics, timed on their own (no allocation, device only)
    dout = torch.zeros(8, dtype=torch.float64, device=f"cuda:{local}")
    G.diagnostics_noalloc(ctx, dout)
    torch.cuda.synchronize()
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    for _ in range(20):
        G.diagnostics_noalloc(ctx, dout)
    d1.record(stream)
    torch.cuda.synchronize()
    diag_ms = d0.elapsed_time(d1) / 20
    # per-kernel breakdown (events between kernel groups, no graph)
    prof = G.step_profiled(ctx, 3)
    parts = {k: v / 3.0 for k, v in prof.items()}
    upd = (parts["update_c2p_pred"] + parts["update_c2p_corr"]) / 2.0
    flux = sum(parts[f"flux_x{d}_{s}"] for d in (1, 2, 3) for s in ("pred", "corr")) / 6.0
    kernels_ms = {k: round(v, 4) for k, v in parts.items()}
    fp64_peak = G.peak_probe(local, True)
    fp32_peak = G.peak_probe(local, False)
    hbm_peak, hbm_peak_src = measured_peaks()
    # Roofline of the dominant kernel, the stage update + inversion (k_update):
    # bound by the FP64 pipe (GB300: 1/64 of the FP32 rate).  achieved = the
    # algorithmic FP64 flops of one launch (the oracle's operation count of the
    # inversion at the Newton steps per zone measured in this run, plus the RK
    # accumulation) / the launch's CUDA-event time measured above.
    dd = {k: diag[k] - d_w0[k] for k in ("nr_iters", "n_nr", "n_floor", "n_steps")}
    stages = 2.0 * zones * max(dd["n_steps"], 1)
    newton_per_zone = dd["nr_iters"] / stages
    flops_zone = C2P_FIXED_FLOPS + C2P_NEWTON_FLOPS * newton_per_zone + RK_FLOPS
    ach_tf = flops_zone * zones / (upd * 1e-3) / 1e12
    upd_bytes = 0.5 * (UPDATE_BYTES_PER_ZONE["pred"] + UPDATE_BYTES_PER_ZONE["corr"])
    upd_gbs = upd_bytes * zones / (upd * 1e-3) / 1e9
    sha = update_sources_sha()
    traffic = UPDATE_DRAM_BYTES_PER_ZONE * zones if sha == UPDATE_SOURCES_SHA else None
    roofline = {"bound": "alu", "kernel": "k_update<float> (stage update + FP64 inversion, mixed path)",
                "achieved": ach_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach_tf / FP64_PEAK_TFLOPS,
                "traffic": traffic,
                "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz (unit counts and maximum clock); "
                               f"FMA-chain probe on this GPU {fp64_peak:.3f} TFLOP/s",
                "ms_per_launch": upd, "zones_per_launch": zones,
                "flops_per_zone_stage": flops_zone, "newton_steps_per_zone_stage": newton_per_zone,
                "floored_zones_per_stage": dd["n_floor"] / stages,
                "flops_source": "oracle operation counter: inversion 171 + 61 per Newton step, RK 18",
                "traffic_source": (f"ncu dram bytes of one 96^3 launch, {UPDATE_DRAM_BYTES_PER_ZONE} B/zone, "
                                   "scaled by zone count")
                                  if traffic else f"kernel sources changed since the ncu capture (sha {sha})",
                "hbm": {"bytes_per_zone_stage": upd_bytes, "achieved": upd_gbs, "peak": hbm_peak, "unit": "GB/s",
                        "frac": upd_gbs / hbm_peak, "peak_source": hbm_peak_src}}
    hbm_step = HBM_BYTES_PER_ZONE_CYCLE["mixed"] * zones / (ms_step * 1e-3) / 1e9
    gpu_launches = 21 * args.steps
    # ---- e2e through the public API with pinned host buffers: every step
    # copies its inputs in from pinned host memory, steps, and copies its
    # result back.  The state a step needs is its conserved vector U (the
    # primitives are re-derived from it on the device, grmhd_set_state_u), so
    # U alone moves each way; the full state (P and U) is timed beside it.
    # Sequential: one context, one step after another.  Pipelined: three
    # contexts, each driven by its own host thread, so that one context's
    # copies overlap the others' steps (the copies of a step and the step
    # itself still run in order).
    e2e = None
    if not args.no_e2e:
        Ph = torch.empty((8, n, n, n), dtype=torch.float64, pin_memory=True).numpy()
        Uh = torch.empty((9, n, n, n), dtype=torch.float64, pin_memory=True).numpy()
        G.get_state(ctx, Ph, Uh)
        t_0, dt_0 = diag["t"], diag["dt"]
        bytes_full = int(Ph.nbytes + Uh.nbytes)
        bytes_u = int(Uh.nbytes)

        def e2e_full(c, P_host, U_host, k):
            torch.cuda.set_device(local)
            t, dt = t_0, dt_0
            for _ in range(k):
                G.set_state(c, P_host, U_host, t, dt)
                G.step(c, 1)
                _, _, t, dt = G.get_state(c, P_host, U_host)

        def e2e_steps(c, P_host, U_host, k):
            torch.cuda.set_device(local)  # a worker thread starts on device 0
            t, dt = t_0, dt_0
            for _ in range(k):
                G.set_state_u(c, U_host, t, dt)
                G.step(c, 1)
                _, t, dt = G.get_state_u(c, U_host)

        ne = 3
        timed_full = []
        for fn in (e2e_full, e2e_steps):
            G.set_state(ctx, Ph, Uh, t_0, dt_0)
            barrier()
            torch.cuda.synchronize()
            t_start = time.perf_counter()
            fn(ctx, Ph, Uh, ne)
            torch.cuda.synchronize()
            timed_full.append(max_over_ranks(time.perf_counter() - t_start, dist, "cuda"))
        full_seq_value = aggregate_value(zones, ne, world, timed_full[0] * 1e3)
        seq_value = aggregate_value(zones, ne, world, timed_full[1] * 1e3)
        # the pipelined form: more contexts, each with its own pinned buffers
        nctx = 3
        extra = [make_ctx(G.MIXED) for _ in range(nctx - 1)]
        bufs = [(ctx, Ph, Uh)]
        for c in extra:
            Pb = torch.empty((8, n, n, n), dtype=torch.float64, pin_memory=True).numpy()
            Ub = torch.empty((9, n, n, n), dtype=torch.float64, pin_memory=True).numpy()
            Pb[...] = Ph
            Ub[...] = Uh
            G.set_state(c, Pb, Ub, t_0, dt_0)
            e2e_steps(c, Pb, Ub, 1)  # first use of its graph and staging
            bufs.append((c, Pb, Ub))
        npipe = 4
        errors = []

        def worker(c, Pb, Ub):
            try:
                e2e_steps(c, Pb, Ub, npipe)
            except BaseException as exc:  # re-raised below: a failed worker voids the number
                errors.append(exc)

        workers = [threading.Thread(target=worker, args=b) for b in bufs]
        barrier()
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        for w in workers:
            w.start()
        for w in workers:
            w.join()
        if errors:
            raise errors[0]
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t_start, dist, "cuda")
        e2e = {"value": aggregate_value(zones, nctx * npipe, world, el * 1e3), "unit": "zone-cycles/s",
               "h2d_bytes_per_step": bytes_u, "d2h_bytes_per_step": bytes_u,
               "steps": nctx * npipe,
               "path": f"grmhd_set_state_u(host U; the primitives re-derived on the device) + grmhd_step + "
                       f"grmhd_get_state(host U) per step, pinned buffers; {nctx} contexts driven by {nctx} "
                       f"host threads, so one context's copies overlap the others' steps",
               "sequential": {"value": seq_value, "steps": ne,
                              "path": "the same calls on one context, one step after another"},
               "full_state_sequential": {"value": full_seq_value, "steps": ne,
                                         "h2d_bytes_per_step": bytes_full, "d2h_bytes_per_step": bytes_full,
                                         "path": "grmhd_set_state(host P and U) + grmhd_step + "
                                                 "grmhd_get_state(host P and U), one context"}}
        for c in extra:
            c.close()
        del Ph, Uh, bufs
    ctx.close()
    torch.cuda.synchronize()
    # ---- the plain FP64 step beside it
    fp64 = None
    if not args.no_fp64:
        k64 = args.fp64_steps or max(3, args.steps // 4)
        c64 = make_ctx(G.FP64)
        ms64, _ = timed(c64, k64, min(args.warmup, 3), False)
        prof64 = G.step_profiled(c64, 1)
        fp64 = {"value": aggregate_value(zones, k64, world, ms64), "unit": "zone-cycles/s", "steps": k64,
                "ms_per_step": ms64 / k64,
                "hbm_frac_of_measured": HBM_BYTES_PER_ZONE_CYCLE["fp64"] * zones / (ms64 / k64 * 1e-3) / 1e9 / hbm_peak,
                "kernels_ms": {k: round(v, 3) for k, v in prof64.items()}}
        c64.close()
    # ---- batched ensemble (independent tori, one launch per kernel class)
    ensemble = None
    if world == 1 and not args.no_ensemble:
        ensemble = run_ensemble(G, torch, stream, local)
        ensemble["small_tori"] = run_ensemble(
            G, torch, stream, local, steps=20, n=96, shapes=SMALL_SHAPES,
            workload="96 small FM tori (64x64x1, 96x64x1, 128x64x1, 64x64x4), same parameter draws, where a loop "
                     "of per-torus step graphs is bound by launches")
    # ---- stand-alone inversion throughput and its FP64 fraction
    c2p = None
    if world == 1 and not args.no_window:
        c2p = run_con2prim(G, torch, stream, local)
    # ---- mixed vs FP64 over the first 200 steps of the 128^3 torus
    window = None
    if world == 1 and not args.no_window:
        window = run_window(G, torch, stream, local)
    # ---- the same torus as phi slabs on this GPU (the multi-GPU layout)
    slabs = theta_slabs = None
    if world == 1 and not args.no_slabs:
        slabs = run_slabs(G, torch, local, n)
        theta_slabs = run_theta_slabs(G, torch, local)
        # a grid whose step is short enough that launches and host reads count
        theta_slabs["small_grid"] = run_theta_slabs(G, torch, local, n1=256, n2=256, steps=40, counts=(2, 4))
    # ---- the 256^3 workload's (gamma, beta_0) grid, and its FP64-vs-mixed window
    variants = window256 = None
    if world == 1 and not args.no_window:
        variants = run_variants(G, torch, stream, local, n)
        window256 = run_window(G, torch, stream, local, n=n, steps=100, every=10, pert=0.04, seed=3)
    # ---- the same workload with PPM faces
    ppm = None
    if world == 1 and not args.no_ppm:
        ppm = run_ppm(G, torch, stream, local, n)
    # ---- learned Newton start: training, inversions, the 256x192x192 step
    mlp = None
    if world == 1 and not args.no_mlp:
        mlp = run_mlp(G, torch, stream, local, fp32_peak)
    # ---- CPU baseline: the oracle on the host cores (rank 0 only, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        zc, dt, desc = oracle_sample_run(n, 2, 2, 0)
        cpu = {"value": zc, "unit": "zone-cycles/s", "cores": 1, "kind": "oracle", "sample": desc}
        # the same oracle on all host cores at once (the single-core figure is the baseline)
        zca, cores, desca = oracle_all_cores(n, 2, 2)
        cpu["all_cores"] = {"value": zca, "unit": "zone-cycles/s", "cores": cores, "kind": "oracle",
                            "sample": desca}
        # the small configurations: 64x64x1 in full (20 steps), 128^3 as a 128x128x4 phi-slab sample
        cpu["configs"] = {
            "64x64x1 (gamma 13/9, r_out 40 M, 20 steps)": oracle_timed(64, 64, 1, 20, 13.0 / 9.0, 40.0, 1),
            "128^3 sample: 128x128x4 (gamma 4/3, r_out 1000 M, 2 steps)": oracle_timed(128, 128, 4, 2, 4.0 / 3.0,
                                                                                    1000.0, 2),
        }
    if rank == 0:
        line = {
            "metric": "zone-cycles/s at 256^3 (FP64 vs mixed, same GB300); % of HBM roofline",
            "value": value, "unit": "zone-cycles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 fluxes + f64 U/inversion", "data": "synthetic",
            "config": workload_config(n),
            "hbm_roofline": {"bytes_per_zone_cycle": HBM_BYTES_PER_ZONE_CYCLE["mixed"], "achieved_gbs": hbm_step,
                             "peak_gbs": hbm_peak, "frac_of_measured": hbm_step / hbm_peak,
                             "frac_of_nominal_7900": hbm_step / 7900.0},
            "roofline": roofline,
            "peaks_probe_tflops": {"fp64": fp64_peak, "fp32": fp32_peak},
            "kernels_ms_per_step": kernels_ms,
            "fp64_step": fp64,
            "ensemble": ensemble,
            "learned_start": mlp,
            "phi_slabs": slabs,
            "theta_slabs": theta_slabs,
            "mixed_vs_fp64_window": window,
            "mixed_vs_fp64_window_256": window256,
            "variants_256": variants,
            "con2prim": c2p,
            "ppm_step": ppm,
            "diagnostics_ms": diag_ms,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "windows": windows,
            "diagnostics_after_bench": dict(
                {k: diag[k] for k in ("t", "dt", "mdot", "eta", "divb_max", "n_fail", "n_fixed", "nr_iters", "n_nr",
                                      "n_entropy_beta", "n_floor")},
                barycentric_radius_r80=bary[0], barycentric_ms_host_sync=bary_ms),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
