#!/usr/bin/env python
"""Throughput benchmark of the N-body hot path on GB300.

Workload (one "step" = one KDK leapfrog step of the whole hot path: staging,
all-pairs mixed-precision force with fused potential, kicks and drift, float64
energy / momentum reduction): a seeded Plummer sphere of N = 65 536 bodies,
G = 1, eps = 0.005, dt = 5e-4, masses 1/N. Metric: body-body interactions per
second (N^2 per force evaluation). Beside it: the plain FP64 GPU path on the
same state, the force error of the mixed path against the FP64 CPU oracle on
sampled bodies, the force kernel's fraction of the FP32-pipe roofline, an
end-to-end figure through the host-memory entry point, and the oracle itself
timed on this host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs an independent system (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "body-body interactions/s, mixed vs FP64 path at ≤1e-4 force err; % FP32 roofline"
UNIT = "interactions/s"
WORKLOAD = dict(n=65536, G=1.0, eps=0.005, dt=5e-4, seed=2)
# float32-pipe operations per interaction in the mixed force kernel:
# 3 FADD (d) + 3 FFMA (s^2) + 3 FMUL (m/s, 1/s^2, m/s^3) + 3 FFMA (a) + 1 FADD (phi); MUFU.RSQ not counted
OPS_PER_INTERACTION = 13
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
L2_FLUSH_BYTES = 256 << 20
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "force_mixed_n65536_full.md")
FORCE_SRC = os.path.join(ROOT, "paper_2511_02655_gb300", "csrc", "force_kernels.cu")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-aux", action="store_true", help="skip the other workloads' short measurements")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(value, dist=None, device=None):
    """Max of a float over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, max_seconds):
    """Whole-job throughput: units all ranks processed / the slowest rank's time."""
    return world * float(units_per_rank) / max_seconds


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: BENCH_CLOCKS_DIR if set (to keep them), else the system temp directory
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_per_launch():
    """DRAM bytes per force launch from the committed ncu summary, if it still matches the source."""
    try:
        text = open(TRAFFIC_FILE).read()
        nbytes = re.search(r"DRAM bytes per launch \(.*?\): (\d+)", text)
        src_sha = re.search(r"Kernel source SHA-256 \(.*?\): ([0-9a-f]{64})", text)
        sha = hashlib.sha256(open(FORCE_SRC, "rb").read()).hexdigest()
        if not nbytes or not src_sha or src_sha.group(1) != sha:
            return None
        return float(nbytes.group(1))
    except Exception:
        return None


def rel_force_error(a, a_ref, guard=1e-3):
    """|a - a_ref| / |a_ref| per body, floored at guard * rms(|a_ref|) (cancellation guard)."""
    import numpy as np
    nrm = np.linalg.norm(a_ref, axis=1)
    rms = float(np.sqrt(np.mean(nrm ** 2)))
    return np.linalg.norm(a - a_ref, axis=1) / np.maximum(nrm, guard * rms)


def cpu_baseline(x, m, G, eps, a_gpu, budget_s=12.0):
    """The oracle (as it stands) on a bounded sample: forces of k seeded bodies against all N."""
    import numpy as np

    import oracle
    from paper_2511_02655_gb300 import inputs
    n = len(m)
    threads = oracle.default_threads()
    probe = inputs.sample_indices(n, 128, seed=99)
    t0 = time.perf_counter()
    oracle.forces_at(x, m, probe, G=G, eps=eps, threads=threads)
    per_body = (time.perf_counter() - t0) / len(probe)
    k = int(max(256, min(n, budget_s / max(per_body, 1e-9))))
    idx = inputs.sample_indices(n, k, seed=7)
    t0 = time.perf_counter()
    a_ref, _ = oracle.forces_at(x, m, idx, G=G, eps=eps, threads=threads)
    dt = time.perf_counter() - t0
    err = rel_force_error(a_gpu[idx], a_ref)
    # the same oracle on one host thread, on a smaller sample (about 2 s)
    k1 = int(max(16, min(n, 2.0 / max(per_body * threads, 1e-9))))
    idx1 = inputs.sample_indices(n, k1, seed=8)
    t0 = time.perf_counter()
    oracle.forces_at(x, m, idx1, G=G, eps=eps, threads=1)
    dt1 = time.perf_counter() - t0
    base = {"value": k * n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"FP64 direct-sum forces of {k} seeded bodies against all {n} (1 force pass, "
                      f"{k * n:.3e} interactions, {dt:.1f} s)",
            "one_thread": {"value": k1 * n / dt1, "sample": f"{k1} seeded bodies against all {n}, {dt1:.1f} s"}}
    return base, {"median": float(np.median(err)), "max": float(err.max()), "bodies": int(k)}


def _event_time(fn, stream, nvtx=None):
    """CUDA-event seconds of fn() on stream; the launches sit in NVTX range `nvtx` (for ncu filters)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if nvtx:
        torch.cuda.nvtx.range_push(nvtx)
    e0.record(stream)
    fn()
    e1.record(stream)
    if nvtx:
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def aux_measurements(dev):
    """The other workloads, each measured briefly (rank 0, one GPU): CUDA-event times around
    nbody_step / nbody_adjoint calls, initialisation and autotuning excluded."""
    import numpy as np
    import torch

    import paper_2511_02655_gb300 as nb
    from paper_2511_02655_gb300 import inputs
    stream = torch.cuda.current_stream()
    out = {}
    # two Plummer spheres, N = 1 048 576, eps = 0.002, dt = 5e-4, mixed
    n = 1048576
    x, v, m = inputs.two_spheres(n, seed=3)
    ctx = nb.nbody_init(G=1.0, eps=0.002, dt=5e-4, precision=nb.MIXED, n=n)
    xt, vt, mt = (torch.from_numpy(t).to(dev) for t in (x, v, m))
    at = torch.empty_like(xt)
    nb.nbody_forces(ctx, xt, mt, at, None, with_phi=False)
    nb.nbody_profile(ctx, True)
    k = 3
    sec = _event_time(lambda: nb.nbody_step(ctx, xt, vt, mt, at, True, k), stream, "aux_two_spheres")
    kms, kl = nb.nbody_kernel_time(ctx, 0)
    nb.nbody_sync(ctx)
    out["two_spheres_1m"] = {"interactions_per_s": float(n) * n * k / sec, "steps": k,
                             "force_kernel_ms": kms / kl, "tuning": nb.nbody_get_tuning(ctx)}
    ctx.close()
    del xt, vt, mt, at
    # ensemble: 512 Plummer systems, N log-uniform in [64, 16384], eps = 0.01, dt = 1e-3
    ens = inputs.ensemble(512, seed=4)
    off = [int(o) for o in ens.offsets]
    pairs = float((np.diff(ens.offsets).astype(np.float64) ** 2).sum())
    ctx = nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=nb.MIXED, offsets=off, energy_every=50,
                        flags=nb.FLAG_GRAPH)
    xt, vt, mt = (torch.from_numpy(t).to(dev) for t in (ens.x, ens.v, ens.m))
    at = torch.empty_like(xt)
    log = torch.empty((1, 512, 9), dtype=torch.float64, device=dev)
    nb.nbody_forces(ctx, xt, mt, at, None, with_phi=False)
    nb.nbody_step(ctx, xt, vt, mt, at, True, 50, log)  # captures the graph
    l0 = nb.nbody_launch_count(ctx)
    sec = _event_time(lambda: nb.nbody_step(ctx, xt, vt, mt, at, True, 50, log), stream, "aux_ensemble")
    nb.nbody_sync(ctx)
    launches = nb.nbody_launch_count(ctx) - l0
    ctx.close()
    # the same systems as 512 separate FP64 contexts, one launch sequence per system, 1 step
    ctxs, bufs = [], []
    for s_ in range(512):
        b, e = off[s_], off[s_ + 1]
        c1 = nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=nb.FP64, n=e - b, block=128, i_per_thread=1,
                           j_tile=128)
        xs, vs, ms = (torch.from_numpy(np.ascontiguousarray(t[b:e])).to(dev) for t in (ens.x, ens.v, ens.m))
        a1 = torch.empty_like(xs)
        nb.nbody_forces(c1, xs, ms, a1, None, with_phi=False)
        ctxs.append(c1), bufs.append((xs, vs, ms, a1))

    def per_system():
        for c1, (xs, vs, ms, a1) in zip(ctxs, bufs):
            nb.nbody_step(c1, xs, vs, ms, a1, True, 1)

    sec64 = _event_time(per_system, stream, "aux_ensemble_fp64")
    for c1 in ctxs:
        c1.close()
    out["ensemble_512"] = {"mixed_graph_interactions_per_s": pairs * 50 / sec, "steps": 50,
                           "fp64_per_system_interactions_per_s": pairs / sec64,
                           "graph_over_fp64_per_system": (pairs * 50 / sec) / (pairs / sec64),
                           "pairs_per_step": pairs, "launches_per_50_steps": int(launches)}
    # the paper's own system: Lennard-Jones gas, 10 000 particles, 2500 KDK steps with the total
    # energy reduced every step, reflecting walls (reduced units, density 0.05, T = 2, dt = 5e-3)
    n, steps = 10000, 2500
    x, v, m, box = inputs.lj_gas(n, seed=9)
    lj = {}
    for prec, flags, name in ((nb.MIXED, nb.FLAG_GRAPH, "mixed_graph"), (nb.FP64, 0, "fp64")):
        ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=prec, n=n, dt=5e-3, box=box, energy_every=1,
                            flags=flags)
        xt, vt, mt = (torch.from_numpy(a).to(dev) for a in (x, v, m))
        at = torch.empty_like(xt)
        logt = torch.empty((steps, 1, 9), dtype=torch.float64, device=dev)
        if flags:  # capture once on a copy of the state, replay on the real one
            x2, v2, a2 = xt.clone(), vt.clone(), torch.empty_like(xt)
            nb.nbody_step(ctx, x2, v2, mt, a2, False, steps, logt)
            nb.nbody_sync(ctx)
            x2.copy_(xt), v2.copy_(vt)
            xt, vt, at = x2, v2, a2
        sec = _event_time(lambda: nb.nbody_step(ctx, xt, vt, mt, at, False, steps, logt), stream, f"aux_lj_{name}")
        nb.nbody_sync(ctx)
        e = logt.cpu().numpy()[:, 0, 0]
        lj[name] = {"seconds": sec, "interactions_per_s": float(n) * n * (steps + 1) / sec,
                    "energy_drift_max_rel": float(np.abs(e - e[0]).max() / abs(e[0]))}
        ctx.close()
    out["paper_lj_gas_10000x2500"] = dict(lj, context="paper (Sec. VI): 19.02 s median, RAJA, 4x A100, FP64, "
                                                      "with energy reduction; other hardware, context only")
    # adjoint: N = 16384 Plummer, 200 KDK steps, dt = 1e-3, checkpoints every 20, loss sum |x_T - t|^2
    n = 16384
    x, v, m = inputs.plummer(n, seed=5)
    t = torch.from_numpy(inputs.targets(n, seed=6)).to(dev)
    for prec, name in ((nb.MIXED, "adjoint_16384_mixed"), (nb.FP64, "adjoint_16384_fp64")):
        ctx = nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=prec, n=n)
        xt, vt, mt = (torch.from_numpy(a).to(dev) for a in (x, v, m))
        xs, vs, at = xt.clone(), vt.clone(), torch.empty_like(xt)
        nb.nbody_step(ctx, xs, vs, mt, at, False, 200)
        lam = 2 * (xs - t)
        nb.nbody_adjoint(ctx, xt, vt, mt, 200, 20, lam, torch.zeros_like(vs))  # tunes the VJP tiling
        sec = _event_time(lambda: nb.nbody_adjoint(ctx, xt, vt, mt, 200, 20, lam, torch.zeros_like(vs)), stream,
                          f"aux_{name}")
        nb.nbody_sync(ctx)
        out[name] = {"seconds": sec, "steps": 200, "checkpoint_every": 20,
                     "force_passes": 200 + 1 + (10 - 1) * (20 - 1), "vjp_passes": 201}
        ctx.close()
    return out


def run_reference(args):
    """The CPU oracle on this host's cores, on the same workload: each step is a bounded sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2511_02655_gb300 import inputs
    w = WORKLOAD
    x, v, m = inputs.plummer(w["n"], seed=w["seed"])
    n = w["n"]
    threads = oracle.default_threads()
    probe = inputs.sample_indices(n, 64, seed=98)
    t0 = time.perf_counter()
    oracle.forces_at(x, m, probe, G=w["G"], eps=w["eps"], threads=threads)
    per_body = (time.perf_counter() - t0) / len(probe)
    per_step_budget = max(0.05, 150.0 / max(1, args.steps + args.warmup))
    k = int(max(32, min(n, per_step_budget / max(per_body, 1e-9))))
    for s in range(args.warmup):
        oracle.forces_at(x, m, inputs.sample_indices(n, k, seed=1000 + s), G=w["G"], eps=w["eps"], threads=threads)
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.forces_at(x, m, inputs.sample_indices(n, k, seed=2000 + s), G=w["G"], eps=w["eps"], threads=threads)
    dt = time.perf_counter() - t0
    value = k * n * args.steps / dt
    sample = f"each step: FP64 direct-sum forces of {k} seeded bodies against all {n}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "plummer N=65536 eps=0.005 (CPU oracle, sampled rows)",
                                             "n_bodies": n, "sample_bodies_per_step": k},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_2511_02655_gb300 as nb
    from paper_2511_02655_gb300 import inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    nb.load()  # fails loudly without the built library
    w = WORKLOAD
    n, G, eps, dt = w["n"], w["G"], w["eps"], w["dt"]
    x, v, m = inputs.plummer(n, seed=w["seed"] + rank)
    K, W = args.steps, max(3, args.warmup)
    stream = torch.cuda.current_stream()

    # ---- mixed path: init + autotune (excluded from timing, as the paper excludes initialisation)
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=nb.MIXED, n=n, energy_every=1)
    tuning = nb.nbody_get_tuning(ctx)
    xt, vt, mt = (torch.from_numpy(t).to(dev) for t in (x, v, m))
    at = torch.empty_like(xt)
    nb.nbody_forces(ctx, xt, mt, at, None, with_phi=False)
    a0 = at.cpu().numpy()
    E0 = nb.nbody_energy(ctx, xt, vt, mt).cpu().numpy()[0, 0]
    log = torch.empty((W + K, 1, 9), dtype=torch.float64, device=dev)
    for k in range(W):
        nb.nbody_step(ctx, xt, vt, mt, at, True, 1, log[k:k + 1])
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = nb.nbody_launch_count(ctx)
    nb.nbody_profile(ctx, True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("bench_timed")  # lets ncu select the timed launches (--nvtx-include)
    for k in range(K):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        ev[k][0].record(stream)
        nb.nbody_step(ctx, xt, vt, mt, at, True, 1, log[W + k:W + k + 1])
        ev[k][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    launches = nb.nbody_launch_count(ctx) - launches0
    force_ms, force_launches = nb.nbody_kernel_time(ctx, 0)
    nb.nbody_profile(ctx, False)
    nb.nbody_sync(ctx)
    total_ms = reduce_max(sum(a.elapsed_time(b) for a, b in ev), pg, dev)
    interactions = float(n) * n
    value = whole_job_rate(interactions * K, world, total_ms * 1e-3)
    elog = log.cpu().numpy()[:, 0, 0]
    drift = float(np.abs(elog - E0).max() / abs(E0))

    # ---- dominant kernel vs its roofline (FP32 pipe, derived from SM count and max clock)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    kernel_s = force_ms * 1e-3 / max(1, force_launches)
    achieved = OPS_PER_INTERACTION * interactions / kernel_s / 1e12
    peak = sms * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    traffic = traffic_per_launch()

    # ---- plain FP64 GPU path on the same state (a few steps)
    ctx64 = nb.nbody_init(G=G, eps=eps, dt=dt, precision=nb.FP64, n=n)
    x64, v64, a64 = xt.clone(), vt.clone(), torch.empty_like(xt)
    nb.nbody_forces(ctx64, x64, mt, a64, None, with_phi=False)
    nb.nbody_step(ctx64, x64, v64, mt, a64, True, 1)
    k64 = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("fp64_path")
    e0.record(stream)
    nb.nbody_step(ctx64, x64, v64, mt, a64, True, k64)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    fp64_value = interactions * k64 / (e0.elapsed_time(e1) * 1e-3)
    ctx64.close()

    # ---- end to end through the host-memory entry point (pinned buffers, copies inside the timing):
    # a context with the same tiling that replays its step as a CUDA graph; L2 flushed between
    # steps outside the timing, each call timed on the host clock (it returns after its sync)
    ke = max(3, min(K, 50))
    ctx_h = nb.nbody_init(G=G, eps=eps, dt=dt, precision=nb.MIXED, n=n, energy_every=1, flags=nb.FLAG_GRAPH,
                          block=tuning["block"], i_per_thread=tuning["i_per_thread"], j_tile=tuning["j_tile"],
                          slice=tuning["slice"], variant=tuning["variant"])
    xh = xt.cpu().pin_memory()
    vh = vt.cpu().pin_memory()
    mh = mt.cpu().pin_memory()
    ah = at.cpu().pin_memory()
    lh = torch.empty((1, 1, 9), dtype=torch.float64).pin_memory()
    for _ in range(W):
        nb.nbody_step_host(ctx_h, xh, vh, mh, ah, True, 1, lh)
    e2e_s = 0.0
    for _ in range(ke):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nb.nbody_step_host(ctx_h, xh, vh, mh, ah, True, 1, lh)
        e2e_s += time.perf_counter() - t0
    e2e_s = reduce_max(e2e_s, pg, dev)
    ctx_h.close()
    e2e = {"value": whole_job_rate(interactions * ke, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": n * 10 * 8, "d2h_bytes_per_step": n * 9 * 8 + 9 * 8,
           "call": "nbody_step_host (1 KDK step per call, pinned host x, v, m, a in; x, v, a, energy out; "
                   "step replayed as a CUDA graph; L2 flushed between calls, outside the timing)"}

    # ---- CPU oracle on this host (rank 0, N = 1 only), which also gives the force error
    base, ferr = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, ferr = cpu_baseline(x, m, G, eps, a0)
    ctx.close()
    aux = None
    if rank == 0 and world == 1 and not args.no_aux:
        del xt, vt, mt, at, flush
        torch.cuda.empty_cache()
        aux = aux_measurements(dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": "Plummer sphere N=65536 (seeded), G=1, eps=0.005, dt=5e-4, 1 KDK step + energy/"
                            "momentum reduction per step, mixed precision",
                "n_bodies": n, "precision": "f32 pair arithmetic, compensated f32 tile sums, f64 slice sums, "
                                            "f64 state and reductions",
                "l2": "flushed (256 MiB write) between timed steps",
                "tuning": tuning,
                "fp64_path_interactions_per_s": fp64_value,
                "mixed_over_fp64": value / world / fp64_value,
                "force_err_vs_oracle": ferr,
                "energy_drift_max_rel": drift,
                "interactions_per_step": interactions,
            },
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s (FP32 pipe)",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_force_mixed", "ops_per_interaction": OPS_PER_INTERACTION,
                         "kernel_ms": kernel_s * 1e3,
                         "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {SM_MAX_MHZ:.0f} MHz"},
            "cpu_baseline": base,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": int(launches),
            "aux": aux,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
