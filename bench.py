"""Benchmark of the fast-multipole BEM matvec (and the GMRES solve it drives) on GB300.

Default workload: silver-like sphere a=1, eps=-8.5+0.3i, k0 a=0.5, icosphere subdivision 7
(163842 Nystrom nodes), one x-polarised plane wave along +z, plain FP64 method.  One step = one
fast-multipole matvec y = A x through every pass (source densities, P2M, M2M, M2L + L2L, near
field + L2P + self blocks).  value = nodes x right-hand sides per second of device time, inputs
resident in HBM; L2 is flushed (256 MiB write) before every timed step.

Also reported: e2e (same metric through the C ABI with pinned host buffers and the host<->device
copies inside the timed region), the roofline of the dominant kernel, the solve time to a 1e-4
relative residual, and the FP64 CPU oracle timed on a bounded sample of rows (cpu_baseline).

``--impl reference`` times the FP64 CPU oracle instead (the reference arm of this comparison).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import fmbem_inputs as fi  # noqa: E402

WORKLOADS = {
    "silver_sphere_s7": dict(mesh=lambda: fi.icosphere(7), eps=[1.0, -8.5 + 0.3j], mu=[1.0, 1.0], k0=0.5, n_rhs=1,
                             desc="silver-like sphere a=1, eps=-8.5+0.3i, k0 a=0.5, icosphere subdivision 7"),
    "sphere_s4": dict(mesh=lambda: fi.icosphere(4), eps=[1.0, 2.25], mu=[1.0, 1.0], k0=1.0, n_rhs=1,
                      desc="dielectric sphere a=1, eps=2.25, k0 a=1, icosphere subdivision 4"),
    "torus_512x128": dict(mesh=lambda: fi.torus(), eps=[1.0, -10 + 0.4j], mu=[1.0, 1.0], k0=1.5, n_rhs=128,
                          desc="torus R=1 r=0.25 512x128 grid, eps=-10+0.4i, k0 R=1.5, 128 plane waves"),
}
METRIC = "FMM-BEM matvec points*RHS/s"
UNIT = "points*RHS/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="silver_sphere_s7", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rhs_batch(n_rhs):
    if n_rhs == 1:
        return np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]], dtype=np.complex128)
    return fi.plane_wave_batch(n_rhs // 2, seed=3)


# ------------------------------------------------------------------------------- CPU oracle
def oracle_rows_rate(wl, rows_per_call, calls, seed=2):
    """FP64 oracle: rows of the dense operator per second on a bounded sample."""
    import oracle
    V, F, D = wl["mesh"]()
    o = oracle.Oracle(V, F, D, wl["eps"], wl["mu"], wl["k0"])
    dirs, pols = rhs_batch(wl["n_rhs"])
    x = o.plane_wave_rhs(dirs, pols)
    times = []
    for c in range(calls):
        rows = fi.sample_rows(o.N, rows_per_call, seed=seed + c)
        t = time.perf_counter()
        o.matvec_rows(x, rows)
        times.append(time.perf_counter() - t)
    return o.N, times, oracle.num_threads()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    rows = 512 if wl["n_rhs"] == 1 else 64
    N, _, _ = oracle_rows_rate(wl, rows, 1)  # warm-up / build
    for _ in range(max(0, args.warmup - 1)):
        oracle_rows_rate(wl, rows, 1)
    _, times, cores = oracle_rows_rate(wl, rows, args.steps)
    t = sum(times)
    value = rows * args.steps * wl["n_rhs"] / t
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * t / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload, nodes=N, n_rhs=wl["n_rhs"], desc=wl["desc"],
                            step=f"{rows} seeded node rows of the dense FP64 operator (all 6 result entries)"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                                  sample=f"{rows} rows x {args.steps} steps of the {N}-node dense operator"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm))


# ------------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1211_7177_gb300 as fm

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    wl = WORKLOADS[args.workload]
    prec = fm.FP64 if args.precision == "fp64" else fm.FP32
    V, F, D = wl["mesh"]()
    t0 = time.perf_counter()
    g = fm.FMBEM(V, F, D, wl["eps"], wl["mu"], wl["k0"], p=args.p, leaf_size=args.leaf, profile_phases=1)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = g.tree_info()
    N, nr = g.N, wl["n_rhs"]
    dirs, pols = rhs_batch(nr)
    b = g.plane_wave_rhs(dirs, pols)
    x = b.clone()
    y = torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        g.matvec(x, y, precision=prec)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-phase times of one matvec (events recorded inside the library on this stream)
    phases = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        phases.append(g.last_matvec_times())
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(bb) for a, bb in ev]
    ms_step = sum(ms) / len(ms)
    if world > 1:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * N * nr / (ms_step * 1e-3)

    # e2e through the C ABI: pinned host x -> device, matvec, device -> pinned host y
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        x.copy_(xh, non_blocking=True)
        step()
        yh.copy_(y, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0.record(stream)
        x.copy_(xh, non_blocking=True)
        step()
        yh.copy_(y, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_val = world * N * nr / (statistics.mean(e2e_ms) * 1e-3)
    nbytes = x.numel() * 16

    # roofline of the dominant kernel (phase with the largest share)
    keys = ["p2m", "m2m", "m2l_l2l", "near_l2p_self"]
    avg = {kk: statistics.mean(ph[kk] for ph in phases) for kk in keys}
    dom = max(keys, key=lambda kk: avg[kk])
    p = args.p
    cols = 3 * nr
    n_dom = len(wl["eps"])
    peaks = {"fp64": 1.2e12, "fp32": 74.6e12}
    if dom == "m2l_l2l":
        flops = 8.0 * p ** 4 * cols * info["ff_pairs"] * n_dom
        name = "k_down (M2L + L2L)"
    elif dom == "near_l2p_self":
        flops = info["near_pairs"] * n_dom * (NEAR_PAIR + NEAR_RHS * nr)
        name = "k_near (P2P + L2P + self)"
    else:
        flops = None
        name = dom
    achieved = flops / (avg[dom] * 1e-3) if flops else None
    peak = peaks[args.precision]
    roof = dict(kernel=name, bound="alu", achieved=achieved / 1e12 if achieved else None, peak=peak / 1e12,
                unit="TFLOP/s", frac=(achieved / peak) if achieved else None, traffic=None,
                peak_source=f"measured {args.precision.upper()} FMA throughput on GB300 (self-written probe)",
                phase_ms=avg)

    solve = None
    if not args.no_solve:
        xs = torch.zeros_like(b)
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        _, its, rr, st = g.solve(b, xs, tol=1e-4, max_iter=500)
        torch.cuda.synchronize()
        solve = dict(tol=1e-4, ms=1e3 * (time.perf_counter() - s0), iters=int(its.max()), relres=float(rr.max()),
                     status=int(st), precision="fp64")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rows = 1024 if nr == 1 else 64
        Nn, times, cores = oracle_rows_rate(wl, rows, 2)
        cpu = dict(value=rows * nr / min(times), unit=UNIT, cores=cores, kind="oracle",
                   sample=f"{rows} seeded node rows of the {Nn}-node dense FP64 operator, best of 2")

    launches_per_step = 3 + (info["l_max"] - 2) + (info["l_max"] - 1)
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms_step, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64" if args.precision == "fp64" else "f32", data="synthetic",
                config=dict(workload=args.workload, desc=wl["desc"], nodes=N, n_rhs=nr, p=p, leaf_size=args.leaf,
                            tree=info, parallelism=f"replicas x{world}", l2="flushed (256 MiB write) before each step",
                            setup_s=setup_s, wall_s=wall),
                e2e=dict(value=e2e_val, unit=UNIT, h2d_bytes_per_step=nbytes, d2h_bytes_per_step=nbytes),
                roofline=roof, cpu_baseline=cpu, solve=solve, gpu_launches=launches_per_step * args.steps,
                clocks=clk)
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


# flops per (near pair, domain): geometry and kernel scalars, and per right-hand side
NEAR_PAIR = 21
NEAR_RHS = 103


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
