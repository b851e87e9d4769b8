"""Throughput benchmark of the fused semiclassical-LBM step on one GB300.

Workload: 3D porous medium 256^3 on the D3V19 lattice (Boolean spheres of
radius 6, porosity 0.7, seed 1), Fermi-Dirac weight (theta = 1/270, mu = 1),
tau = 0.8, E_x = 1e-6, B_z = 1e-3, explicit Lorentz forcing term; populations
stored as FP16 deviations (FP32 collision).  A step is one fused
stream-collide-force pass over the whole box; the state (1.2 GB) is larger
than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the same metric instead (a deliberately slow baseline).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(n=256, radius=6.0, porosity=0.7, seed=1, Ex=1e-6, Bz=1e-3, tau=0.8, dims=None)


def box_dims():
    """(nx, ny, nz) of the box: n^3, or the --dims override (profiling runs)."""
    return tuple(WORKLOAD["dims"]) if WORKLOAD["dims"] else (WORKLOAD["n"],) * 3


def workload_name(n: int) -> str:
    box = f"{n}^3" if not WORKLOAD["dims"] else "x".join(str(d) for d in WORKLOAD["dims"])
    return (f"porous-3d-{box} D3V19 FD(theta=1/270,mu=1) spheres r=6 porosity=0.7 seed=1, "
            "tau=0.8 E_x=1e-6 B_z=1e-3 force=term")

# DRAM traffic per 256^3 launch of the step kernel (dram__bytes_read.sum +
# dram__bytes_write.sum): an ncu capture of one full-size launch of the bench
# workload (three metrics, one pass); keyed by storage, with the hash of the
# kernel source it was taken on, and reported as null once the source has
# changed.
NCU_TRAFFIC = {"f16": (1361035776, "b3004de8ecc87443"), "f32": (2679074000, "897e5af381bb943b")}

FALLBACK_HBM_GBS = 6800.0


def kernel_source_hash(storage: str = "f16") -> str:
    """Hash of the step kernel's source for one storage with comments and
    blank lines removed (a comment edit does not change the kernel the
    counters were taken on)."""
    h = hashlib.sha256()
    for f in ("lbm_step.cuh", "lbm_device.cuh", "lbm_internal.h", f"lbm_step_{storage}.cu"):
        with open(os.path.join(ROOT, "paper_1710_09472_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.samples = []
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for line in (out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def summary(self):
        if not getattr(self, "samples", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        smax = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, name in enumerate(names):
                if s[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def max_over_ranks(times, world: int, device):
    """Each rank's timings -> the element-wise maximum over the ranks of the
    initialised process group (the slowest replica sets the job time)."""
    if world <= 1:
        return list(times)
    import torch
    import torch.distributed as dist

    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def make_geometry():
    from paper_1710_09472_gb300 import workloads as wl

    nx, ny, nz = box_dims()
    mask, count = wl.boolean_obstacles((nz, ny, nx), WORKLOAD["radius"], WORKLOAD["porosity"], WORKLOAD["seed"])
    return mask, count


def run_gpu(args, rank, world):
    import numpy as np
    import torch

    from paper_1710_09472_gb300.build import build
    from paper_1710_09472_gb300.lbm import LBM

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0:
        build()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        build()
    dev = torch.device("cuda", local)
    mask, count = make_geometry()
    n = WORKLOAD["n"]
    dims = box_dims()
    E = (WORKLOAD["Ex"], 0.0, 0.0)
    B = (0.0, 0.0, WORKLOAD["Bz"])
    mask_d = torch.from_numpy(mask.reshape(-1)).to(dev)
    stream = torch.cuda.current_stream(dev)

    def timed_forward(storage):
        sim = LBM("D3V19", dims, WORKLOAD["tau"], E=E, B=B, storage=storage, force="term", stream=stream)
        sim.set_geometry(mask_d)
        sim.init_equilibrium()
        sim.step(args.warmup)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        l0 = sim.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        launches = sim.launch_count() - l0
        info = sim.info()
        rho = torch.empty(sim.N, device=dev)
        j = torch.empty(3 * sim.N, device=dev)
        tot = sim.moments(rho, j)
        return sim, ms, launches, info, (rho, j, tot)

    # primary: FP16-deviation storage.  The clock sampler runs across both timed
    # legs and their set-up (the GPU is busy throughout), so that a short timed
    # region still has samples under the same load.
    with ClockSampler(local) as clk:
        sim16, ms16, launches16, info, m16 = timed_forward("f16")
        sim16.close()
        sim32, ms32, launches32, info32, m32 = timed_forward("f32")
        sim32.close()
    clocks = clk.summary()

    # forward + adjoint: lbm_adjoint over T steps (loss = mean x-current after
    # the last step), checkpoints every K steps, per-cell dL/dE in FP64
    T_adj, K_adj = args.adjoint_steps, args.adjoint_checkpoint
    sim = LBM("D3V19", dims, WORKLOAD["tau"], E=E, B=B, storage="f16", force="term", stream=stream)
    sim.set_geometry(mask_d)
    sim.init_equilibrium()
    n_fluid_a = sim.info()["n_fluid"]
    wj = torch.zeros(3 * sim.N, dtype=torch.float32, device=dev)
    wj[: sim.N] = 1.0 / n_fluid_a
    dE = torch.empty(3 * sim.N, dtype=torch.float64, device=dev)
    sim.adjoint(T_adj - 1, T_adj, None, wj, K_adj, dL_dE=dE)  # warm-up (allocations, clocks)
    sim.init_equilibrium()
    torch.cuda.synchronize()
    l0 = sim.launch_count()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    adj = sim.adjoint(T_adj - 1, T_adj, None, wj, K_adj, dL_dE=dE)
    a1.record(stream)
    torch.cuda.synchronize()
    ms_adj = a0.elapsed_time(a1)
    adj_launches = sim.launch_count() - l0
    adj_stats = sim.adjoint_stats()
    sim.close()

    # whole-job through the public API with pinned host buffers
    N = dims[0] * dims[1] * dims[2]
    mask_h = torch.from_numpy(mask.reshape(-1)).pin_memory()
    rho_h = torch.ones(N, dtype=torch.float32).pin_memory()
    u_h = torch.zeros(3 * N, dtype=torch.float32).pin_memory()
    rho_out = torch.empty(N, dtype=torch.float32).pin_memory()
    j_out = torch.empty(3 * N, dtype=torch.float32).pin_memory()
    sim = LBM("D3V19", dims, WORKLOAD["tau"], E=E, B=B, storage="f16", force="term", stream=stream)
    sim.set_geometry(mask_h)
    sim.init_equilibrium(rho_h, u_h)
    sim.step(args.warmup)
    sim.moments(rho_out, j_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_geometry(mask_h)
    sim.init_equilibrium(rho_h, u_h)
    sim.step(args.steps)
    sim.moments(rho_out, j_out)  # synchronises
    e2e_s = time.perf_counter() - t0
    sim.close()

    def rel(a, b):
        den = float(torch.max(torch.abs(b)))
        return float(torch.max(torch.abs(a - b))) / den if den > 0 else 0.0

    err_rho = rel(m16[0], m32[0])
    err_j = rel(m16[1], m32[1])

    # max over ranks
    ms16, ms32, e2e_s, ms_adj = max_over_ranks([ms16, ms32, e2e_s, ms_adj], world, dev)
    n_fluid = info["n_fluid"]
    Q = 19
    peak, peak_kind = hbm_peak()

    def mlups(ms):
        return world * N * args.steps / (ms * 1e-3) / 1e6

    def roof(ms, b):
        per_launch_ms = ms / args.steps
        alg = 2 * Q * b * n_fluid
        achieved = alg / (per_launch_ms * 1e-3) / 1e9
        return achieved, alg

    ach16, alg16 = roof(ms16, 2)
    ach32, alg32 = roof(ms32, 4)
    src_hash = kernel_source_hash("f16")

    def traffic_of(storage):
        tr = NCU_TRAFFIC.get(storage)
        ok = tr and tr[1] == kernel_source_hash(storage) and box_dims() == (256, 256, 256)
        return tr[0] if ok else None

    traffic = traffic_of("f16")
    result = {
        "metric": "MLUPS",
        "value": round(mlups(ms16), 1),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms16 / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f16-deviation storage, f32 collision",
        "data": "synthetic",
        "config": {"workload": workload_name(n), "storage": "f16-deviation (2^12 scale), FP32 collision",
                   "cells": N, "fluid_cells": n_fluid, "spheres": count, "parallelism": f"replicas x{world}",
                   "l2": f"state {2 * Q * N / 1e9:.2f} GB > 129 MB L2; no flush needed"},
        "mflups": round(world * n_fluid * args.steps / (ms16 * 1e-3) / 1e6, 1),
        "roofline": {"bound": "hbm", "achieved": round(ach16, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(ach16 / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "k_step_rows<D3V19,f16,term>", "alg_bytes_per_launch": alg16},
        "fp32": {"value": round(mlups(ms32), 1), "unit": "MLUPS", "ms_per_step": round(ms32 / args.steps, 5),
                 "roofline": {"bound": "hbm", "achieved": round(ach32, 1), "peak": peak, "unit": "GB/s",
                              "frac": round(ach32 / peak, 4), "traffic": traffic_of("f32"),
                              "alg_bytes_per_launch": alg32}},
        "fwd_adjoint": {
            "value": round(world * N * T_adj / (ms_adj * 1e-3) / 1e6, 1), "unit": "MLUPS",
            "steps": T_adj, "checkpoint_every": K_adj, "ms_per_step": round(ms_adj / T_adj, 5),
            "cost_vs_forward_step": round((ms_adj / T_adj) / (ms16 / args.steps), 3),
            "schedule": adj_stats["schedule"], "states_kept": adj_stats["states"],
            "forward_steps": adj_stats["forward_steps"],
            "what": ("one lbm_adjoint call: the forward steps of its checkpoint schedule and T reverse steps "
                     "(FP64 per-cell dL/dE, dL/dB, dL/dtau); loss = mean x-current after the last step; "
                     "storage f16-deviation"),
            "launches": int(adj_launches), "dL_dtau": adj["dL_dtau"], "dL_dBz": float(adj["dL_dB"][2])},
        "fp16_vs_fp32": {"rho_rel_linf": err_rho, "j_rel_linf": err_j, "after_steps": args.warmup + args.steps},
        "e2e": {"value": round(world * N * args.steps / e2e_s / 1e6, 1), "unit": "MLUPS",
                "h2d_bytes_per_step": int((N + 4 * N + 12 * N) / args.steps),
                "d2h_bytes_per_step": int((4 * N + 12 * N) / args.steps),
                "what": "set_geometry + init_equilibrium from pinned host buffers, K steps, moments to pinned host"},
        "gpu_launches": int(launches16),
        "clocks": clocks,
        "kernel_source": src_hash,
    }
    if not args.no_extra:
        result["adjoint_replayed"] = adjoint_replayed(mask_d, dims, E, B, dev, stream, ms16 / args.steps)
        result["other_lattices"] = other_lattices(mask, dev, stream, peak, args.warmup)
    if args.adjoint_512 > 0:
        result["adjoint_512"] = adjoint_512(args.adjoint_512, dev, stream)
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(mask)
    return result


def _time_steps(sim, steps, warmup, stream):
    import torch

    sim.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def adjoint_replayed(mask_d, dims, E, B, dev, stream, fwd_ms):
    """Forward + adjoint over T = 1000 steps with the segment schedule
    (checkpoints every 32 steps, each segment replayed), loss = mean x-current
    after the last step, per-cell FP64 dL/dE: the cost of a step including
    the replay, against one forward step of the same storage."""
    import torch

    from paper_1710_09472_gb300.lbm import LBM

    T, K = 1000, 32
    sim = LBM("D3V19", dims, WORKLOAD["tau"], E=E, B=B, storage="f16", force="term", stream=stream)
    sim.set_geometry(mask_d)
    sim.init_equilibrium()
    n_fluid = sim.info()["n_fluid"]
    wj = torch.zeros(3 * sim.N, dtype=torch.float32, device=dev)
    wj[: sim.N] = 1.0 / n_fluid
    dE = torch.empty(3 * sim.N, dtype=torch.float64, device=dev)
    sim.adjoint(K - 1, K, None, wj, K, dL_dE=dE)  # allocations
    sim.init_equilibrium()
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    sim.adjoint(T - 1, T, None, wj, K, dL_dE=dE)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1)
    st = sim.adjoint_stats()
    sim.close()
    return {"steps": T, "checkpoint_every": K, "schedule": st["schedule"], "forward_steps": st["forward_steps"],
            "reverse_steps": st["reverse_steps"], "ms_per_step": round(ms / T, 5),
            "cost_vs_forward_step": round((ms / T) / fwd_ms, 3), "storage": "f16-deviation"}


def other_lattices(mask, dev, stream, peak, warmup):
    """Throughput of the other lattices through the same kernels, and of the
    1D thermal model (fourth-order EDF on D1V7): MLUPS and the fraction of
    the HBM roofline at 2 Q b bytes per fluid-cell update."""
    import torch

    from paper_1710_09472_gb300.lbm import LBM, Thermal

    out = {}
    n = WORKLOAD["n"]
    steps = 200
    mask_d = torch.from_numpy(mask.reshape(-1)).to(dev)
    box = box_dims()
    # (D1V3 boxes are at most 2^20 cells, whose state fits the 129 MB L2, so
    # they have no HBM figure)
    # the local chemical-potential model (per-cell thetabar) runs on its own
    # row-staged instantiation (run-time row stride)
    for vel, dims, storage, local in (("D3V27", box, "f16", False), ("D3V27", box, "f32", False),
                                      ("D3V19", box, "f16", True)):
        sim = LBM(vel, dims, WORKLOAD["tau"], E=(WORKLOAD["Ex"], 0.0, 0.0), B=(0.0, 0.0, WORKLOAD["Bz"]),
                  storage=storage, force="term", stream=stream)
        sim.set_geometry(mask_d)
        if local:
            sim.set_local_mu(True)
        sim.init_equilibrium()
        ms = _time_steps(sim, steps, warmup, stream)
        info = sim.info()
        b = 4 if storage == "f32" else 2
        alg = 2 * info["Q"] * b * info["n_fluid"]
        gbs = alg / (ms * 1e-3) / 1e9
        key = f"{vel} {storage} {'local-mu ' if local else ''}porous " + "x".join(str(d) for d in dims)
        out[key] = {"MLUPS": round(info["N"] / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms, 5),
                    "roofline_frac": round(gbs / peak, 4), "achieved_GBs": round(gbs, 1)}
        sim.close()
    nx = 1 << 24
    for storage in ("f32", "f16"):
        t = Thermal("D1V7", nx, 0.8, E=1e-5, order=4, storage=storage, stat="fd", theta=0.3, mu=1.0, stream=stream)
        t.init()
        ms = _time_steps(t, steps, warmup, stream)
        b = 4 if storage == "f32" else 2
        gbs = 2 * t.Q * b * nx / (ms * 1e-3) / 1e9
        out[f"thermal D1V7 order 4 {storage} periodic {nx}"] = {
            "MLUPS": round(nx / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms, 5),
            "roofline_frac": round(gbs / peak, 4), "achieved_GBs": round(gbs, 1)}
        t.close()
    return out


def adjoint_512(T: int, dev, stream):
    """Forward + full adjoint on the 512^3 porous box (spheres r = 10, porosity
    0.65, seed 5; E_x = 2e-6, B_z = 5e-4, tau 0.8, FP16-deviation storage):
    loss = mean x-current after T steps, dL/dE(x) per cell, with the kept
    forward states limited to what fits 180 GB of device memory together with
    the adjoint fields, the context's own states and dL/dE (the binomial
    schedule when the segment schedule does not fit)."""
    import torch

    from paper_1710_09472_gb300 import workloads as wl
    from paper_1710_09472_gb300.lbm import LBM

    n = 512
    mask, count = wl.boolean_obstacles((n, n, n), 10.0, 0.65, 5)
    sim = LBM("D3V19", (n, n, n), 0.8, E=(2e-6, 0.0, 0.0), B=(0.0, 0.0, 5e-4), storage="f16", force="term",
              stream=stream)
    sim.set_geometry(torch.from_numpy(mask.reshape(-1)).to(dev))
    del mask
    sim.init_equilibrium()
    N = sim.N
    n_fluid = sim.info()["n_fluid"]
    wj = torch.zeros(3 * N, dtype=torch.float32, device=dev)
    wj[:N] = 1.0 / n_fluid
    dE = torch.empty(3 * N, dtype=torch.float64, device=dev)
    state = sim.adjoint_stats()["state_bytes"]
    # an adjoint field: FP32 lambda plus one FP32 per link (the state holds one FP16 per link)
    lam_field = 4 * 19 * N + 2 * max(0, state - 2 * 19 * N) + 1024
    fixed = 2 * lam_field + 2 * state + dE.numel() * (8 + 4) + wj.numel() * 4  # dL/dE: FP64 + FP32 partials
    budget = 180 * 10**9 - fixed - 4 * 10**9  # margin: CUDA context, library scratch, torch buffers
    sim.set_memory_budget(budget)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = sim.adjoint(T - 1, T, None, wj, 0, dL_dE=dE)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st = sim.adjoint_stats()
    out = {"T": T, "seconds": round(dt, 2), "ms_per_step": round(dt * 1e3 / T, 3), "schedule": st["schedule"],
           "states_kept": st["states"], "state_gb": round(state / 1e9, 3),
           "device_gb_budgeted": round((st["states"] * state + fixed) / 1e9, 1),
           "forward_steps": st["forward_steps"], "reverse_steps": st["reverse_steps"],
           "dL_dtau": res["dL_dtau"], "dL_dBz": float(res["dL_dB"][2]), "spheres": count, "fluid_cells": n_fluid,
           "dL_dE_sum_x": float(dE[:N].sum())}
    sim.close()
    return out


def _oracle_sample(mask, box: int):
    """A box^3 sub-block of the same geometry, periodic, at rest."""
    import numpy as np

    sub = np.ascontiguousarray(mask[:box, :box, :box])
    return sub


def cpu_baseline(mask, target_s: float = 12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload."""
    import numpy as np

    import oracle

    box = 96
    sub = _oracle_sample(mask, box)
    shape = sub.shape
    m = oracle.Model("D3V19", "fd", 1.0 / 270.0, 1.0, tau=WORKLOAD["tau"], E=(WORKLOAD["Ex"], 0, 0),
                     B=(0, 0, WORKLOAD["Bz"]), force="term")
    f = m.init_equilibrium(shape, sub, np.ones(shape))
    t0 = time.perf_counter()
    m.step(shape, sub, f, 1)
    one = time.perf_counter() - t0
    steps = max(1, min(200, int(target_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    m.step(shape, sub, f, steps)
    dt = time.perf_counter() - t0
    cells = box ** 3
    return {"value": round(cells * steps / dt / 1e6, 3), "unit": "MLUPS", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{box}^3 sub-box of the same sphere packing (periodic), {steps} steps, FP64 C with OpenMP"}


def run_reference(args, rank, world):
    """The oracle on the host cores as the reference arm: each step is one
    oracle time step over a 64^3 sub-box of the same workload."""
    import numpy as np

    import oracle

    if rank != 0:
        return None
    mask, count = make_geometry()
    box = 64
    sub = _oracle_sample(mask, box)
    shape = sub.shape
    m = oracle.Model("D3V19", "fd", 1.0 / 270.0, 1.0, tau=WORKLOAD["tau"], E=(WORKLOAD["Ex"], 0, 0),
                     B=(0, 0, WORKLOAD["Bz"]), force="term")
    f = m.init_equilibrium(shape, sub, np.ones(shape))
    m.step(shape, sub, f, args.warmup)
    t0 = time.perf_counter()
    m.step(shape, sub, f, args.steps)
    dt = time.perf_counter() - t0
    v = round(box ** 3 * args.steps / dt / 1e6, 3)
    sample = f"{box}^3 sub-box of the same sphere packing (periodic), FP64 C oracle with OpenMP"
    return {"metric": "MLUPS", "value": v, "unit": "MLUPS", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(WORKLOAD["n"]), "sample": sample},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--adjoint-checkpoint", type=int, default=0,
                    help="checkpoint_every of lbm_adjoint (0: schedule sized to the free memory)")
    ap.add_argument("--n", type=int, default=256, help="box edge (256 is the benchmark; smaller for profiling)")
    ap.add_argument("--dims", default="", help="nx,ny,nz box instead of n^3 (smaller cases for profiling)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the replayed-adjoint and other-lattice keys (profiling runs)")
    ap.add_argument("--adjoint-512", type=int, default=0,
                    help="also run the 512^3 forward + full adjoint over this many steps within 180 GB (0 = off)")
    args = ap.parse_args()
    WORKLOAD["n"] = args.n
    if args.dims:
        WORKLOAD["dims"] = [int(v) for v in args.dims.split(",")]
        if len(WORKLOAD["dims"]) != 3:
            ap.error("--dims takes nx,ny,nz")
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    res = run_gpu(args, rank, world)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
