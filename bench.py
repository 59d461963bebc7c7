"""Benchmark of the fast-multipole BEM matvec (and the GMRES solve it drives) on GB300.

Default workload: silver-like sphere a=1, eps=-8.5+0.3i, k0 a=0.5, icosphere subdivision 7
(163842 Nystrom nodes), one x-polarised plane wave along +z, plain FP64 method, truncation p=10
(the FMM tolerance 1e-5 class: 4.7e-6 relative L2 against the dense FP64 oracle on 2048 rows).
One step = one fast-multipole matvec y = A x through every pass (source densities, P2M, M2M,
M2L + L2L, near field + L2P + self blocks).  value = nodes x right-hand sides per second of device
time, inputs resident in HBM; L2 is flushed (256 MiB write) before every timed step.

Also reported: e2e (same metric through the C ABI with pinned host buffers and the host<->device
copies inside the timed region), the roofline of the dominant kernel, the same matvec in FP32
arithmetic, the solve time to a 1e-4 relative residual for the plain FP64 solve and for the
FP32-inner / FP64-outer refined solve, and the FP64 CPU oracle timed on a bounded sample of rows
(cpu_baseline).

The default run adds a ``batched`` object: the batched mixed-precision form on the torus
R=1, r=0.25 (512x128 grid, 65536 nodes, eps=-10+0.4i, k0 R=1.5) with 128 plane waves -- the
128-RHS matvec with M2L + L2L on the tensor cores in the BF16x3 form (bf16 hi/lo split operands,
three products per step; device time and e2e, per-phase rooflines; the TF32 form's time beside it),
the FP64 single-RHS matvec on the same mesh, the plain FP64 single-RHS solve and the batched solve
(BF16x3 inner GMRES, FP64-operator true residual) to 1e-4, and the FP64 oracle on sampled rows
(timed, with the matvec error and the batched solution's residual against the dense operator).
``--workload torus_512x128`` runs the 128-right-hand-side batch as the main line instead.

It also adds ``uneven_batch``: 256 seeded particles (spheroids, tori, split rings of 2k-60k
triangles, 4 plane waves each) whose products run in ONE persistent kernel launch with a device
work queue, timed beside the same products issued one problem at a time, with the oracle's error
on sampled rows of 16 of the particles.

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
                             p=10, desc="silver-like sphere a=1, eps=-8.5+0.3i, k0 a=0.5, icosphere subdivision 7"),
    "silver_sphere_s6": dict(mesh=lambda: fi.icosphere(6), eps=[1.0, -8.5 + 0.3j], mu=[1.0, 1.0], k0=0.5, n_rhs=1,
                             p=10, desc="silver-like sphere a=1, eps=-8.5+0.3i, k0 a=0.5, icosphere subdivision 6 "
                                        "(the profiling case)"),
    "sphere_s4": dict(mesh=lambda: fi.icosphere(4), eps=[1.0, 2.25], mu=[1.0, 1.0], k0=1.0, n_rhs=1, p=8,
                      desc="dielectric sphere a=1, eps=2.25, k0 a=1, icosphere subdivision 4"),
    "torus_512x128": dict(mesh=lambda: fi.torus(), eps=[1.0, -10 + 0.4j], mu=[1.0, 1.0], k0=1.5, n_rhs=128, p=8,
                          desc="torus R=1 r=0.25 512x128 grid, eps=-10+0.4i, k0 R=1.5, 128 plane waves"),
}
METRIC = "FMM-BEM matvec points*RHS/s"
UNIT = "points*RHS/s"
# flops per (near pair, domain): geometry (double-float difference, |r|, n.r, w = n x r) and the
# kernel scalars g, c; and per (near pair, domain, right-hand side): u = w x v + (n.r) v and two
# complex FMAs per row -- counted from the near-field kernels' source (FADD/FMUL = 1, FFMA = 2,
# each transcendental = 1)
NEAR_PAIR = 52
NEAR_RHS = 78
# FP64 with fewer than 4 right-hand sides reads g and c from the near-field cache built at create:
# per pair only r, w = n x r and n.r remain (14 flops, shared by both domains), and the scatterer
# domain's bracket is the background's plus s r (6 FFMA per RHS instead of u's 30 flops): per
# (pair, domain) 7 + 69 per right-hand side, averaged over the two domains
NEAR_PAIR_CACHED = 7
NEAR_RHS_CACHED = 69
PEAK_TFLOPS = {"fp64": 1.2, "fp32": 74.6}  # measured FMA throughput on GB300 (self-written probe)
TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense TF32 : BF16 tensor-core rate


class nvtx_range:
    """An NVTX range around a timed region (named for profiler filters: ncu --nvtx-include name/)."""

    def __init__(self, name):
        self.name = name

    def __enter__(self):
        import torch
        torch.cuda.nvtx.range_push(self.name)

    def __exit__(self, *a):
        import torch
        torch.cuda.nvtx.range_pop()


def tensor_peak_tf32():
    """Dense TF32 tensor-core peak: the measured cuBLAS BF16 burst rate times the nominal ratio."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16, src = float(json.load(f)["bf16_tflops"]), "of measured"
    except (OSError, KeyError, ValueError):
        bf16, src = 1900.0, "of fallback"
    return bf16 * TF32_OVER_BF16, f"{src} BF16 GEMM burst rate x nominal TF32/BF16 ratio 1.1/2.25"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="silver_sphere_s7", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "tf32", "bf16x3"])
    ap.add_argument("--p", type=int, default=0, help="truncation number (0 = the workload's)")
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-impedance", action="store_true", help="skip the impedance-boundary product")
    ap.add_argument("--gradients", action="store_true",
                    help="with the adjoint gradients, also check one vertex against central differences")
    ap.add_argument("--no-gradients", action="store_true",
                    help="skip the adjoint gradients on the torus + sphere differentiation case")
    ap.add_argument("--restart", type=int, default=50, help="GMRES restart length of the timed solves")
    ap.add_argument("--n-rhs", type=int, default=0, help="right-hand sides (0 = the workload's)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched leg (128-RHS torus, BF16x3 tensor-core M2L, FP64-refined solve) of the default run")
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the uneven-batch leg (256 particles in one persistent launch) of the default run")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value, device):
    """The largest of the ranks' values (all ranks get it); the value itself with one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms):
    """Whole-job rate: the units every rank processed in ms milliseconds (the slowest rank's)."""
    return world * units_per_rank / (ms * 1e-3)


def rhs_batch(n_rhs):
    if n_rhs == 1:
        return np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]], dtype=np.complex128)
    return fi.plane_wave_batch(n_rhs // 2, seed=3)


# ------------------------------------------------------------------------------- CPU oracle
def oracle_rows_rate(wl, rows_per_call, calls, seed=2):
    """FP64 oracle: seconds for rows_per_call rows of the dense operator, `calls` times."""
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
    rows = 512 if wl["n_rhs"] == 1 else 32
    N, _, _ = oracle_rows_rate(wl, rows, 1)
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
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
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
def m2l_flops_per_column(p, nr):
    """Algorithmic real flops of one S|R translation of one column: dense p^2 x p^2 complex matrix
    (8 p^4), or, in the rotation form the library uses for p >= 9 with at most 8 right-hand sides,
    an azimuthal phase and a fold into mirror-even/odd halves, a real polar rotation per degree on
    the folded halves (real x complex, 4 flops per entry), the complex coaxial S|R per order block,
    the folded polar rotation back, the unfold and a phase."""
    if p >= 9 and 3 * nr <= 24:
        rot = p * (2 * p * p + 1) // 3     # folded polar entries per rotation
        coax = p * (2 * p * p + 1) // 3    # coaxial entries
        return (4.0 * 2 * rot + 8.0 * coax + 6.0 * 2 * p * p + 4.0 * p * p,
                "rotation form (phase, folded real polar rotation, coaxial S|R, back)")
    return 8.0 * p ** 4, "dense S|R matrices"


def roofline(info, p, nr, n_dom, phases, precision, workload=None):
    """Roofline of the dominant phase of the matvec, and in `phases` the same figures for the near
    field (+ L2P + self) and for M2L + L2L, each against the peak of the arithmetic it runs in."""
    keys = ["p2m", "m2m", "m2l_l2l", "near_l2p_self"]
    avg = {k: statistics.mean(ph[k] for ph in phases) for k in keys}
    arith = "fp32" if precision in ("tf32", "bf16x3") else precision
    alu_peak, alu_src = PEAK_TFLOPS[arith], f"measured {arith.upper()} FMA throughput of GB300 (self-written probe)"
    out = {}
    # M2L + L2L
    tensor = (precision == "bf16x3" and (3 * nr <= 24 or tensor_path(nr))) or (precision == "tf32" and tensor_path(nr))
    if tensor:
        per_col = 8.0 * p ** 4
        if precision == "bf16x3":
            form = "dense S|R on tcgen05, BF16x3 (bf16 hi/lo operands, three products)"
            peak, src = tensor_peak_bf16x3()
        else:
            form = "dense S|R on tcgen05 TF32"
            peak, src = tensor_peak_tf32()
        bound = "tensor"
    else:
        per_col, form = m2l_flops_per_column(p, nr)
        peak, src, bound = alu_peak, alu_src, "alu"
    flops = per_col * 3 * nr * info["ff_pairs"] * n_dom
    ach = flops / (avg["m2l_l2l"] * 1e-3) / 1e12
    out["m2l_l2l"] = dict(kernel=f"M2L + L2L, {form}", bound=bound, achieved=ach, peak=peak, unit="TFLOP/s",
                          frac=ach / peak, ms=avg["m2l_l2l"], algorithmic_flops_per_launch=flops, peak_source=src,
                          traffic=phase_traffic(workload, precision, nr, "m2l_l2l"))
    # near field + L2P + self
    cached = precision == "fp64" and nr < 4
    per_pair, per_rhs = (NEAR_PAIR_CACHED, NEAR_RHS_CACHED) if cached else (NEAR_PAIR, NEAR_RHS)
    flops = info["near_pairs"] * n_dom * (per_pair + per_rhs * nr)
    ach = flops / (avg["near_l2p_self"] * 1e-3) / 1e12
    kern = ("k_near (pair-scalar cache)" if cached else "k_near_rb") if arith == "fp64" else \
        ("k_near_ws" if nr < 4 else "k_near_r + k_near_w" if nr >= 32 else "k_near_w")
    out["near_l2p_self"] = dict(kernel=f"near field + L2P + self ({kern})", bound="alu", achieved=ach, peak=alu_peak,
                                unit="TFLOP/s", frac=ach / alu_peak, ms=avg["near_l2p_self"],
                                algorithmic_flops_per_launch=flops, peak_source=alu_src,
                                traffic=phase_traffic(workload, precision, nr, "near_l2p_self"))
    dom = max(out, key=lambda k: avg[k])
    r = dict(out[dom])
    r.pop("ms")
    r["phase_ms"] = avg
    r["phases"] = out
    return r


def tensor_path(nr):
    """The TF32 matvec runs M2L + L2L on the tensor cores for at least 16 right-hand sides."""
    return 3 * nr >= 48


def launches_per_matvec(lmax, nr, n_dom, precision, p, rotation):
    """Kernels per matvec of the main line's path, as the ncu launch lists under profiles/ show
    them (every domain of a level in one launch):
    - tensor-core path (BF16x3 or TF32, 16 or more RHS, p <= 8): the densities (k_prep_node_major
      for whole blocks of 32 RHS in BF16x3, else k_prep, plus k_dens_node_major when there are
      32 or more), P2M (k_p2m_tc in BF16x3, k_p2m_gemm in TF32), M2M per level 3..l_max
      (k_m2l_tc in BF16x3; k_m2m on the CUDA cores in TF32), k_round_tf32 (TF32), one k_m2l_tc per
      level 2..l_max, and the near field (k_near_r per whole block launch, k_near_w for the rest);
    - otherwise k_prep and P2M; M2M per level 3..l_max (the rotation form: k_m2l_rot* + k_mm_reduce;
      dense: k_m2m); the downward pass: BF16x3 with at most 8 RHS: k_split_bf16, two k_m2l_ofs
      launches and per level a k_l2l_reduce (with a rotation-form L2L on levels 3..l_max);
      else per level a k_l2l_reduce after the M2L (k_m2l_rot* or k_m2l_chunks), with the L2L
      translation as its own launch on levels 3..l_max in the rotation form; one near-field
      kernel."""
    near = 1
    if precision in ("bf16x3", "tf32") and tensor_path(nr) and p <= 8:
        bf3 = precision == "bf16x3"
        prep = 1 if (bf3 and nr % 32 == 0) else (2 if nr >= 32 else 1)
        near = (1 if nr >= 32 else 0) + (1 if nr % 32 else 0)
        return prep + 1 + (lmax - 2) + (0 if bf3 else 1) + (lmax - 1) + near
    m2m = 2 * (lmax - 2) if rotation else (lmax - 2)
    if precision == "bf16x3" and 3 * nr <= 24:
        down = 1 + 2 + 1 + (2 if rotation else 1) * (lmax - 2)
    else:
        down = 2 + (3 if rotation else 2) * (lmax - 2)
    return 2 + m2m + down + near


def run_gradients(fd_check=False):
    """Differentiation case: a silver-like torus (R = 1, r = 0.25, 256 x 64 grid, 32768 triangles,
    eps = -10 + 0.4i) and a dielectric sphere (a = 0.1, eps = 2.5, 1280 triangles) a seeded gap
    above the tube, k0 R = 1.5, one plane wave along -z.  Times the extinction's gradient with
    respect to eps and to every vertex, and the Maxwell-stress force on the sphere with its vertex
    gradient (forward and adjoint FMM solves included: refined, BF16x3-operator inner GMRES and
    FP64-operator true residuals), and with fd_check compares one sphere vertex of the force
    gradient with central differences of full GPU solves."""
    import torch

    import paper_1211_7177_gb300 as fm
    from paper_1211_7177_gb300 import gradients as gr
    opts = dict(solve_precision=fm.BF16X3, inner_tol=1e-3)
    a = 0.1
    (V, F, D), gap, ctr = fi.torus_and_sphere(seed=4, a=a)
    eps, mu, k0 = [1.0, -10 + 0.4j, 2.5], [1.0, 1.0, 1.0], 1.5
    d = np.array([0.0, 0.0, -1.0])
    e = np.array([1.0, 0.0, 0.0], dtype=np.complex128)
    rad = a + 0.5 * gap
    out = dict(nodes=len(V), gap=gap, stress_sphere_radius=rad, solves="refined: BF16x3 inner, FP64 outer, tol 1e-8")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c, de_re, de_im = gr.extinction_eps_gradient(V, F, D, eps, mu, k0, d[None], e[None], j=2, tol=1e-8, **opts)
    torch.cuda.synchronize()
    out["extinction_eps_gradient_s"] = time.perf_counter() - t0
    out["dcext_deps2"] = [float(de_re[0]), float(de_im[0])]
    t0 = time.perf_counter()
    c, gV = gr.extinction_vertex_gradient(V, F, D, eps, mu, k0, d[None], e[None], tol=1e-8, **opts)
    torch.cuda.synchronize()
    out["extinction_vertex_gradient_s"] = time.perf_counter() - t0
    out["cext"] = float(c[0])
    t0 = time.perf_counter()
    Fo, gF = gr.force_vertex_gradient(V, F, D, eps, mu, k0, d, e, ctr, rad, tol=1e-8, **opts)
    torch.cuda.synchronize()
    out["force_vertex_gradient_s"] = time.perf_counter() - t0
    out["force"] = [float(v) for v in Fo]
    if not fd_check:
        return out
    # central difference of the force for one vertex of the sphere (its vertices follow the torus')
    v, h = len(V) - 5, 1e-6
    fd = []
    for sgn in (1, -1):
        Vx = V.copy()
        Vx[v, 2] += sgn * h
        fd.append(gr.force_vertex_gradient(Vx, F, D, eps, mu, k0, d, e, ctr, rad, tol=1e-12, **opts)[0])
    out["force_fd_check"] = dict(vertex=int(v), coordinate="z", adjoint=[float(q) for q in gF[:, v, 2]],
                                 central_difference=[float(q) for q in (fd[0] - fd[1]) / (2 * h)])
    return out


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one matvec phase, from ncu
# captures summarised under profiles/ (launches_*.md: the timed steps' launches, one metric pass,
# caches flushed between kernels), keyed by (workload, precision, n_rhs, phase); each entry
# records the SHA-256 prefixes of the kernel sources it was taken with, and the bench reports null
# once a source has changed.
TRAFFIC = {
    ('silver_sphere_s7', 'fp64', 1, 'p2m'): dict(bytes=2213602816, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'fp64', 1, 'm2m'): dict(bytes=117071872, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'fp64', 1, 'm2l_l2l'): dict(bytes=5563075072, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'fp64', 1, 'near_l2p_self'): dict(bytes=6586166784, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'fp32', 1, 'p2m'): dict(bytes=1114655488, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'fp32', 1, 'm2m'): dict(bytes=58543872, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'fp32', 1, 'm2l_l2l'): dict(bytes=2677159680, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'fp32', 1, 'near_l2p_self'): dict(bytes=466040320, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'bf16x3', 1, 'p2m'): dict(bytes=1114879744, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'bf16x3', 1, 'm2m'): dict(bytes=58574080, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'bf16x3', 1, 'm2l_l2l'): dict(bytes=3223854080, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('silver_sphere_s7', 'bf16x3', 1, 'near_l2p_self'): dict(bytes=466579712, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('torus_512x128', 'bf16x3', 128, 'p2m'): dict(bytes=3513320192, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('torus_512x128', 'bf16x3', 128, 'm2m'): dict(bytes=1576227072, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('torus_512x128', 'bf16x3', 128, 'm2l_l2l'): dict(bytes=4913404416, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
    ('torus_512x128', 'bf16x3', 128, 'near_l2p_self'): dict(bytes=4988141312, src={'fmm.cu': '4618eded26d502e7', 'm2l_tc.cu': 'b48e3b613c191a6f'}),
}


def _src_sha(name):
    import hashlib
    with open(os.path.join(ROOT, "paper_1211_7177_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def phase_traffic(workload, precision, nr, phase):
    t = TRAFFIC.get((workload, precision, nr, phase))
    if t is None:
        return None
    if any(_src_sha(f) != h for f, h in t["src"].items()):
        return None
    return t["bytes"]


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


def gmres_roofline(N, iters, restart, ms_total, matvec_ms):
    """Roofline of the plain FP64 GMRES(m) work outside the products, per Arnoldi step: the
    solve's time less its products (iters Arnoldi products + one true residual per cycle after the
    first -- x0 = 0 makes the first residual b itself -- + the final one), over the algorithmic
    bytes and FP64 flops of the steps it ran.  Step j (slots
    0..j of the basis, b = 96 bytes per node per vector): preconditioner (u_j, the 6 x 6 LU
    factors, z: 2b + 582); classical Gram-Schmidt twice with the second pass delayed: one
    reduction of slots 0..j against u_j and w ((j + 2) b), the norm of w (b), one update pass
    (slots 0..j and w read, v_j and u_{j+1} written: (j + 4) b); FP64 flops (2 (j + 1) + 2 j + 2)
    x 6 complex MACs (8 flops) per node plus the LU solve (288)."""
    b = 96.0
    js = [k % restart for k in range(iters)]
    cycles = (iters + restart - 1) // restart
    step_bytes = sum(582.0 + b * (2 * j + 9) for j in js) * N / max(iters, 1)
    step_flops = sum(48.0 * (4 * j + 4) + 288.0 for j in js) * N / max(iters, 1)
    products = iters + cycles
    over_ms = (ms_total - products * matvec_ms) / max(iters, 1)
    hbm, hsrc = hbm_peak()
    ach_gbs = step_bytes / (over_ms * 1e-3) / 1e9 if over_ms > 0 else None
    ach_tf = step_flops / (over_ms * 1e-3) / 1e12 if over_ms > 0 else None
    t_hbm, t_fp64 = step_bytes / (hbm * 1e9), step_flops / (PEAK_TFLOPS["fp64"] * 1e12)
    return dict(bound="fp64" if t_fp64 > t_hbm else "hbm", ms_per_step=over_ms, products=products,
                bytes_per_step=step_bytes, flops_per_step=step_flops,
                achieved_gbs=ach_gbs, hbm_peak_gbs=hbm, hbm_frac=ach_gbs / hbm if ach_gbs else None,
                achieved_fp64_tflops=ach_tf, fp64_frac=ach_tf / PEAK_TFLOPS["fp64"] if ach_tf else None,
                bound_ms_per_step=1e3 * max(t_hbm, t_fp64),
                peak_source=f"HBM {hsrc} copy bandwidth; FP64 measured FMA throughput (self-written probe)")


def tensor_peak_bf16x3():
    """Effective tensor peak of the BF16x3 form: the measured cuBLAS BF16 burst rate over the three
    bf16 products that carry one algorithmic product."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16, src = float(json.load(f)["bf16_tflops"]), "of measured"
    except (OSError, KeyError, ValueError):
        bf16, src = 1900.0, "of fallback"
    return bf16 / 3, f"{src} BF16 GEMM burst rate / 3 (three bf16 products per algorithmic product)"


def phase_rooflines(info, p, nr, n_dom, N, phases, workload, form="bf16x3"):
    """Per-phase roofline of the batched matvec: near field against the FP32 ALU peak, M2L + L2L
    (algorithmic flops of the dense complex contraction) against the tensor peak of the form
    (BF16x3: the BF16 rate over three; TF32), M2M and P2M against the BF16x3 tensor peak in that
    form (they run on the tensor cores there; the P2M phase also forms the densities, k_prep) and
    against the FP32 ALU peak in the TF32 form."""
    keys = ["p2m", "m2m", "m2l_l2l", "near_l2p_self"]
    avg = {k: statistics.mean(ph[k] for ph in phases) for k in keys}
    tpk, tsrc = tensor_peak_bf16x3() if form == "bf16x3" else tensor_peak_tf32()
    cols = 3 * nr * n_dom
    flops = {
        # per (near pair, domain): the kernel scalars; per (pair, domain, RHS): the bracket and g q
        "near_l2p_self": info["near_pairs"] * n_dom * (NEAR_PAIR + NEAR_RHS * nr),
        # dense S|R in real form on the tensor cores: 8 p^4 per (FF pair, column)
        "m2l_l2l": 8.0 * p ** 4 * info["ff_pairs"] * cols,
        # per (node, side, coefficient, column): a dipole/monopole weight times the basis, 4 complex MACs
        "p2m": 32.0 * N * 2 * p * p * 3 * nr,
        # dense S|S per (child box, column), every box below level 2 has a parent
        "m2m": 8.0 * p ** 4 * max(info["n_boxes"] - 64, 0) * cols,
    }
    out = {}
    for k in keys:
        tensor = k == "m2l_l2l" or (k in ("m2m", "p2m") and form == "bf16x3" and nr >= 16 and 2 * p * p <= 128)
        peak = tpk if tensor else PEAK_TFLOPS["fp32"]
        ach = flops[k] / (avg[k] * 1e-3) / 1e12
        out[k] = dict(bound="tensor" if tensor else "alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                      ms=avg[k], algorithmic_flops=flops[k],
                      traffic=phase_traffic(workload, form, nr, k),
                      peak_source=tsrc if tensor else "measured FP32 FMA throughput of GB300 (self-written probe)")
    return out, avg


def run_batched(args, world, flush):
    """Batched, mixed-precision form on the torus: R = 1, r = 0.25, 512 x 128 grid (65536 nodes),
    eps = -10 + 0.4i, k0 R = 1.5, 128 plane waves (64 Fibonacci directions x 2 polarisations),
    p = 8.  Times the 128-RHS matvec with the M2L on the tensor cores in the BF16x3 form (device
    and e2e; the TF32 form beside it), the
    FP64 single-RHS matvec on the same mesh, the plain FP64 single-RHS solve and the batched solve
    (BF16x3-operator inner GMRES, FP64-operator true residual) to 1e-4; on rank 0 the FP64 oracle
    evaluates sampled rows, timed, giving the matvec error and the solve's residual against the
    dense operator."""
    import torch

    import paper_1211_7177_gb300 as fm
    name = "torus_512x128"
    wl = WORKLOADS[name]
    p, nr, restart = wl["p"], wl["n_rhs"], 100
    rank = dist_env()[0]
    V, F, D = wl["mesh"]()
    t0 = time.perf_counter()
    g = fm.FMBEM(V, F, D, wl["eps"], wl["mu"], wl["k0"], p=p, leaf_size=args.leaf, profile_phases=1,
                 m2l_rotation=1, gmres_restart=restart)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = g.tree_info()
    N, n_dom = g.N, len(wl["eps"])
    dirs, pols = rhs_batch(nr)
    b = g.plane_wave_rhs(dirs, pols)
    noise = torch.from_numpy(fi.random_complex((nr, N, 6), seed=13)).cuda()
    x = b + 0.1 * noise
    del noise
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def time_matvec(xx, yy, prec, steps, warmup, with_phases=True):
        for _ in range(warmup):
            g.matvec(xx, yy, precision=prec)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        ph = []
        with nvtx_range(f"{name}_{ {fm.FP64: 'fp64', fm.FP32: 'fp32', fm.TF32: 'tf32'}.get(prec, 'bf16x3')}_{xx.shape[0]}"):
            for k in range(steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                g.matvec(xx, yy, precision=prec)
                ev[k][1].record(stream)
                if with_phases:
                    ph.append(g.last_matvec_times())
            torch.cuda.synchronize()
        return max_over_ranks(statistics.mean(a.elapsed_time(bb) for a, bb in ev), "cuda"), ph

    ms, phases = time_matvec(x, y, fm.BF16X3, args.steps, args.warmup)
    roof, avg = phase_rooflines(info, p, nr, n_dom, N, phases, name)
    dom = max(avg, key=avg.get)
    out = dict(workload=name, desc=wl["desc"], nodes=N, n_rhs=nr, p=p, leaf_size=args.leaf, tree=info,
               dtype="f32 (M2L + L2L on the tensor cores: bf16 hi/lo split operands, three products, FP32 "
                     "accumulation)", setup_s=setup_s,
               l2="inputs larger than L2 and L2 flushed (256 MiB write) before each step",
               value=job_throughput(N * nr, world, ms), unit=UNIT, ms_per_step=ms, steps=args.steps,
               roofline=dict(roof[dom], kernel=dom), phase_roofline=roof)

    # e2e through the C ABI with host buffers (fmbem_matvec_host): pinned host x -> device,
    # matvec, device -> pinned host y (one chunk of 128 right-hand sides)
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.fill_(float(k))
        e0.record(stream)
        g.matvec_host(xh, yh, precision=fm.BF16X3, stream=stream, sync=False)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    nbytes = x.numel() * 16
    out["e2e"] = dict(value=world * N * nr / (statistics.mean(e2e_ms) * 1e-3), unit=UNIT,
                      h2d_bytes_per_step=nbytes, d2h_bytes_per_step=nbytes)
    y_bf3 = yh.numpy().copy()
    # the TF32 operand form of the same product, for comparison (faster rounding, less accurate)
    ms_tf, _ = time_matvec(x, y, fm.TF32, args.steps, args.warmup, with_phases=False)
    y_tf32 = y.cpu().numpy()
    out["tf32_form"] = dict(value=job_throughput(N * nr, world, ms_tf), unit=UNIT, ms_per_step=ms_tf)

    # the plain method's form on the same mesh: FP64 arithmetic, one right-hand side per matvec
    x1, y1 = x[:1].contiguous(), y[:1].contiguous()
    ms1, _ = time_matvec(x1, y1, fm.FP64, 3, 2, with_phases=False)
    out["fp64_single_rhs"] = dict(value=world * N / (ms1 * 1e-3), unit=UNIT, ms_per_step=ms1)
    out["speedup_vs_fp64_single_rhs"] = out["value"] / out["fp64_single_rhs"]["value"]

    solve = {}
    if not args.no_solve:
        # plain: FP64 GMRES(100) on one right-hand side
        gp = fm.FMBEM(V, F, D, wl["eps"], wl["mu"], wl["k0"], p=p, leaf_size=args.leaf, m2l_rotation=1,
                      gmres_restart=restart)
        b1 = b[:1].contiguous()
        xs1 = torch.zeros_like(b1)
        gp.solve(b1, xs1, tol=1e-4, max_iter=2)  # warm-up: allocates the Krylov basis
        xs1.zero_()
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        _, its, rr, st = gp.solve(b1, xs1, tol=1e-4, max_iter=1000)
        torch.cuda.synchronize()
        t_plain = time.perf_counter() - s0
        solve["plain_fp64_single_rhs"] = dict(tol=1e-4, ms=1e3 * t_plain, iters=int(its.max()), relres=float(rr.max()),
                                              status=int(st), restart=restart,
                                              gmres=gmres_roofline(N, int(its.max()), restart, 1e3 * t_plain, ms1))
        gp.close()
        del gp
        # batched: inner GMRES(100) with the BF16x3 tensor-core operator and a single-precision
        # basis; outer true residual b - A x with the FP64 operator and FP64 vectors, repeated
        # until it is <= 1e-4.  The inner solve goes to a quarter of the target: the BF16x3
        # operator is close enough to the FP64 one that one inner solve then meets the target,
        # and the outer loop takes a single FP64 product (128 columns of FP64 FMM cost about as
        # much as 80 inner iterations)
        itol = 2.5e-5
        gb = fm.FMBEM(V, F, D, wl["eps"], wl["mu"], wl["k0"], p=p, leaf_size=args.leaf, m2l_rotation=1,
                      gmres_restart=restart, solve_precision=fm.BF16X3, inner_tol=itol, outer_precision=fm.FP64)
        xs = torch.zeros_like(b)
        gb.solve(b, xs, tol=1e-4, max_iter=2)  # warm-up
        xs.zero_()
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        _, its, rr, st = gb.solve(b, xs, tol=1e-4, max_iter=2000)
        torch.cuda.synchronize()
        t_b = time.perf_counter() - s0
        solve["batched_bf16x3_inner_fp64_outer"] = dict(
            tol=1e-4, ms=1e3 * t_b, ms_per_rhs=1e3 * t_b / nr, iters=int(its.max()), relres_fp64_true=float(rr.max()),
            status=int(st), restart=restart, inner_tol=itol, n_rhs=nr)
        solve["per_rhs_speedup_vs_plain"] = t_plain / (t_b / nr)
        xs_h = xs.cpu().numpy()
        gb.close()
        del gb
    out["solve"] = solve

    if rank == 0 and not args.no_cpu_baseline:
        # the FP64 CPU oracle on 32 seeded node rows for all 128 right-hand sides (timed: the
        # batched leg's cpu_baseline); the same rows give the tensor-core matvecs' errors and the refined
        # solution's true residual against the dense FP64 operator
        import oracle
        o = oracle.Oracle(V, F, D, wl["eps"], wl["mu"], wl["k0"])
        rows = fi.sample_rows(N, 32, seed=2)
        xh_np = xh.numpy()
        t0 = time.perf_counter()
        yo = o.matvec_rows(xh_np, rows)
        t_or = time.perf_counter() - t0
        out["cpu_baseline"] = dict(value=len(rows) * nr / t_or, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                                   sample=f"{len(rows)} seeded node rows x {nr} RHS of the {N}-node dense FP64 operator")
        err = lambda a: float(np.linalg.norm(a[:, rows] - yo) / np.linalg.norm(yo))
        acc = dict(rows=len(rows), matvec_rel_l2_vs_oracle=err(y_bf3), tf32_form_rel_l2_vs_oracle=err(y_tf32))
        if solve:
            bo = o.plane_wave_rhs(dirs, pols)[:, rows]
            ro = o.matvec_rows(xs_h, rows) - bo
            acc["solve_rel_residual_vs_oracle"] = float(np.linalg.norm(ro) / np.linalg.norm(bo))
        out["accuracy"] = acc
    g.close()
    return out


def run_uneven_batch(args, world, flush):
    """Uneven batch of 256 independent particles (seeded spheroids, tori and split rings of 2k-60k
    triangles, eps from {2.25, -5+0.2i, -12+0.5i}, k0 size 0.3-3, 4 plane waves each): all 256
    products in ONE persistent kernel launch (device work queue, bounded waits), FP32 passes,
    p = 8; beside it the same products issued one problem after another through fmbem_matvec.
    On rank 0 the FP64 oracle evaluates 16 seeded rows of 16 seeded problems (timed: this leg's
    cpu_baseline), giving the batch's error against the dense operators."""
    import torch

    import paper_1211_7177_gb300 as fm
    from paper_1211_7177_gb300.batch import PersistentBatch
    nr = 4
    probs = fi.particle_batch(256, seed=5)
    free0 = torch.cuda.mem_get_info()[0]
    t0 = time.perf_counter()
    hs = [fm.FMBEM(p["V"], p["F"], p["D"], p["eps"], p["mu"], p["k0"], p=8, leaf_size=args.leaf, fp32_only=1)
          for p in probs]
    dirs, pols = fi.plane_wave_batch(2, seed=15)
    xs = [h.plane_wave_rhs(dirs, pols) for h in hs]
    ys = [torch.empty_like(x) for x in xs]
    b = PersistentBatch(hs, nr)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    mem_gb = (free0 - torch.cuda.mem_get_info()[0]) / 2 ** 30
    stream = torch.cuda.current_stream()
    nodes = sum(h.N for h in hs)

    def timed(fn, steps, warmup, name):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with nvtx_range(name):
            for k in range(steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                fn()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        return max_over_ranks(statistics.mean(a.elapsed_time(bb) for a, bb in ev), "cuda")

    ms = timed(lambda: b.matvec(xs, ys), args.steps, args.warmup, "particle_batch")
    y_batch = [y.clone() for y in ys]

    def one_by_one():
        for h, x, y in zip(hs, xs, ys):
            h.matvec(x, y, precision=fm.FP32)

    ms_seq = timed(one_by_one, max(2, args.steps // 4), 2, "particle_one_by_one")
    dev = max(float(torch.linalg.vector_norm(a - c) / torch.linalg.vector_norm(c)) for a, c in zip(y_batch, ys))
    out = dict(workload="particle_batch_256", n_problems=len(hs), nodes_total=nodes, n_rhs=nr,
               triangles=[int(min(len(p["F"]) for p in probs)), int(max(len(p["F"]) for p in probs))],
               p=8, dtype="f32", setup_s=setup_s, device_memory_gb=mem_gb, work_items=b.num_items,
               l2="inputs larger than L2 (1.26 GB of right-hand sides) and L2 flushed before each step",
               value=job_throughput(nodes * nr, world, ms), unit=UNIT, ms_per_step=ms, steps=args.steps,
               one_by_one=dict(value=job_throughput(nodes * nr, world, ms_seq), unit=UNIT, ms_per_step=ms_seq,
                               max_rel_diff_to_batch=dev))
    if dist_env()[0] == 0 and not args.no_cpu_baseline:
        import oracle
        rng = np.random.default_rng(17)
        pick = sorted(rng.choice(len(hs), 16, replace=False).tolist())
        errs, t_or, nrows = [], 0.0, 0
        for i in pick:
            p = probs[i]
            o = oracle.Oracle(p["V"], p["F"], p["D"], p["eps"], p["mu"], p["k0"])
            rows = fi.sample_rows(hs[i].N, 16, seed=i)
            xh = xs[i].cpu().numpy()
            s0 = time.perf_counter()
            yo = o.matvec_rows(xh, rows)
            t_or += time.perf_counter() - s0
            nrows += len(rows)
            errs.append(float(np.linalg.norm(y_batch[i].cpu().numpy()[:, rows] - yo) / np.linalg.norm(yo)))
        out["cpu_baseline"] = dict(value=nrows * nr / t_or, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                                   sample=f"16 seeded rows x {nr} RHS of 16 seeded problems of the batch, dense FP64")
        out["accuracy"] = dict(problems=len(pick), rows_each=16, max_rel_l2_vs_oracle=max(errs),
                               median_rel_l2_vs_oracle=float(np.median(errs)))
    b.close()
    for h in hs:
        h.close()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1211_7177_gb300 as fm

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    wl = WORKLOADS[args.workload]
    p = args.p or wl["p"]
    prec = {"fp64": fm.FP64, "fp32": fm.FP32, "tf32": fm.TF32, "bf16x3": fm.BF16X3}[args.precision]
    V, F, D = wl["mesh"]()
    t0 = time.perf_counter()
    g = fm.FMBEM(V, F, D, wl["eps"], wl["mu"], wl["k0"], p=p, leaf_size=args.leaf, profile_phases=1)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = g.tree_info()
    N, nr = g.N, args.n_rhs or wl["n_rhs"]
    n_dom = len(wl["eps"])
    dirs, pols = rhs_batch(nr)
    b = g.plane_wave_rhs(dirs, pols)
    x = b.clone()
    y = torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(precision, steps, warmup, clocks=False):
        for _ in range(warmup):
            g.matvec(x, y, precision=precision)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if clocks else None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        phases = []
        wall0 = time.perf_counter()
        with nvtx_range(f"{args.workload}_{ {fm.FP64: 'fp64', fm.FP32: 'fp32', fm.TF32: 'tf32'}.get(precision, 'bf16x3')}"):
            for k in range(steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                g.matvec(x, y, precision=precision)
                ev[k][1].record(stream)
                phases.append(g.last_matvec_times())
            torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if world > 1:
            dist.barrier()
        clk = sampler.stop() if sampler else None
        ms = max_over_ranks(statistics.mean(a.elapsed_time(bb) for a, bb in ev), "cuda")
        return ms, phases, wall, clk

    ms_step, phases, wall, clk = timed(prec, args.steps, args.warmup, clocks=True)
    value = job_throughput(N * nr, world, ms_step)
    roof = roofline(info, p, nr, n_dom, phases, args.precision, args.workload)

    # e2e through the C ABI with host buffers (fmbem_matvec_host): pinned host x -> device,
    # matvec, device -> pinned host y, the copies inside the timed region
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        g.matvec_host(xh, yh, precision=prec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0.record(stream)
        g.matvec_host(xh, yh, precision=prec, stream=stream, sync=False)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_val = world * N * nr / (statistics.mean(e2e_ms) * 1e-3)
    nbytes = x.numel() * 16

    other = None
    if not args.no_fp32:
        others = [o for o in ("fp32", "tf32", "bf16x3") if o != args.precision and
                  (o == "fp32" or tensor_path(nr) or (o == "bf16x3" and 3 * nr <= 24))]
        for o in others:
            mso, pho, _, _ = timed({"fp32": fm.FP32, "tf32": fm.TF32, "bf16x3": fm.BF16X3}[o], args.steps, args.warmup)
            other = dict(other or {}, **{o: dict(value=world * N * nr / (mso * 1e-3), ms_per_step=mso,
                                                 roofline=roofline(info, p, nr, n_dom, pho, o, args.workload))})
    if nr > 1:
        # the plain method's form for comparison: FP64 arithmetic, one right-hand side per matvec
        x1, y1 = x[:1].contiguous(), y[:1].contiguous()
        for _ in range(2):
            g.matvec(x1, y1, precision=fm.FP64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            g.matvec(x1, y1, precision=fm.FP64)
        e1.record(stream)
        e1.synchronize()
        ms1 = e0.elapsed_time(e1) / 3
        other = dict(other or {}, fp64_single_rhs=dict(value=world * N / (ms1 * 1e-3), ms_per_step=ms1))

    # the adjoint (transposed) product through the same tree and translations, in the bench's precision
    aprec = {"fp64": fm.FP64, "fp32": fm.FP32, "tf32": fm.TF32, "bf16x3": fm.BF16X3}[args.precision]
    for _ in range(2):
        g.adjoint_matvec(x, y, precision=aprec)
    torch.cuda.synchronize()
    a_ms = []
    for k in range(3):
        flush.fill_(float(k))
        e0.record(stream)
        g.adjoint_matvec(x, y, precision=aprec)
        e1.record(stream)
        e1.synchronize()
        a_ms.append(e0.elapsed_time(e1))
    adjoint = dict(precision=args.precision, ms_per_step=statistics.mean(a_ms),
                   value=world * N * nr / (statistics.mean(a_ms) * 1e-3))

    # the impedance-boundary variant (Section 2.3) on the same mesh: the multipole passes run for
    # the background domain only, the scatterer rows are the local relation of Eq. (2.24)
    impedance = None
    if not args.no_impedance:
        gi = fm.FMBEM(V, F, D, wl["eps"], wl["mu"], wl["k0"], p=p, leaf_size=args.leaf, boundary=fm.IMPEDANCE)
        for _ in range(2):
            gi.matvec(x, y, precision=aprec)
        torch.cuda.synchronize()
        i_ms = []
        for k in range(3):
            flush.fill_(float(k))
            e0.record(stream)
            gi.matvec(x, y, precision=aprec)
            e1.record(stream)
            e1.synchronize()
            i_ms.append(e0.elapsed_time(e1))
        impedance = dict(precision=args.precision, ms_per_step=statistics.mean(i_ms),
                         value=world * N * nr / (statistics.mean(i_ms) * 1e-3))
        gi.close()
        del gi

    solve = None
    if not args.no_solve:
        solve = {}
        if nr == 1:
            kinds = (("plain_fp64", fm.FP64, 0.5e-4), ("fp32_inner_fp64_refined", fm.FP32, 0.5e-4),
                     ("bf16x3_inner_fp64_refined", fm.BF16X3, 0.5e-4))
        else:
            kinds = (("fp32_inner_fp64_refined", fm.FP32, 0.5e-4),) + \
                ((("tf32_inner_fp64_refined", fm.TF32, 1e-2),) if tensor_path(nr) else ())
        for label, sp, itol in kinds:
            # refined solve: FP32 inner GMRES to half the tolerance (TF32 tensor-core M2L: to 1e-2,
            # above the floor its input rounding sets), true residual with the FP64 operator and
            # FP64 vectors
            h2 = fm.FMBEM(V, F, D, wl["eps"], wl["mu"], wl["k0"], p=p, leaf_size=args.leaf, gmres_restart=args.restart,
                          solve_precision=sp, inner_tol=itol, outer_precision=fm.FP64, m2l_rotation=1 if nr > 8 else -1)
            xs = torch.zeros_like(b)
            h2.solve(b, xs, tol=1e-4, max_iter=1000)  # warm-up (allocates the Krylov basis)
            xs.zero_()
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            _, its, rr, st = h2.solve(b, xs, tol=1e-4, max_iter=1000)
            torch.cuda.synchronize()
            solve[label] = dict(tol=1e-4, ms=1e3 * (time.perf_counter() - s0), iters=int(its.max()),
                                relres=float(rr.max()), status=int(st), restart=args.restart, inner_tol=itol)
            if sp == fm.FP64 and nr == 1:
                solve[label]["gmres"] = gmres_roofline(N, int(its.max()), args.restart, solve[label]["ms"], ms_step)
            h2.close()

    gradients = None
    if rank == 0 and args.workload == "silver_sphere_s7" and not args.no_gradients:
        gradients = run_gradients(fd_check=args.gradients)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rows = 1024 if nr == 1 else 16
        Nn, times, cores = oracle_rows_rate(wl, rows, 2)
        cpu = dict(value=rows * nr / min(times), unit=UNIT, cores=cores, kind="oracle",
                   sample=f"{rows} seeded node rows x {nr} RHS of the {Nn}-node dense FP64 operator, best of 2")

    g.close()
    batched = None
    if args.workload == "silver_sphere_s7" and not args.no_batched:
        batched = run_batched(args, world, flush)
    uneven = None
    if args.workload == "silver_sphere_s7" and not args.no_uneven:
        uneven = run_uneven_batch(args, world, flush)

    rotation = p >= 9  # the library's automatic translation form for the main line's handle
    launches_per_step = launches_per_matvec(info["l_max"], nr, n_dom, args.precision, p, rotation)
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms_step, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype={"fp64": "f64", "fp32": "f32", "tf32": "f32 (M2L on TF32 tensor cores)",
                       "bf16x3": "f32 (M2L on tensor cores, bf16 hi/lo split operands)"}[args.precision],
                data="synthetic",
                config=dict(workload=args.workload, desc=wl["desc"], nodes=N, n_rhs=nr, p=p, leaf_size=args.leaf,
                            tree=info, parallelism=f"replicas x{world}",
                            l2="flushed (256 MiB write) before each step", setup_s=setup_s, wall_s=wall),
                e2e=dict(value=e2e_val, unit=UNIT, h2d_bytes_per_step=nbytes, d2h_bytes_per_step=nbytes),
                roofline=roof, other_precision=other, adjoint=adjoint, impedance=impedance, solve=solve,
                gradients=gradients, cpu_baseline=cpu, batched=batched, uneven_batch=uneven,
                gpu_launches=launches_per_step * args.steps, clocks=clk)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
