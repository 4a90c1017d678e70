#!/usr/bin/env python
"""Benchmark of the FR right-hand side on a B300: RHS GDOF/s per RK stage.

Workload (synthetic, seeded): 3D Navier-Stokes on a periodic 96^3 hexahedral
box [0, 2 pi]^3 (884,736 elements), p = 4 (125 solution points, 5 variables,
552.96 M DOF), Taylor-Green initial data (M = 0.1, Re = 1600, Pr = 0.71) plus
a seeded smooth perturbation; LDG beta = 1/2, tau = 0.1.  The paper's own
benchmark is a periodic hexahedral box at p = 2..4 (Sec. 6); its meshes are
not published and this box stands in for them.

One step = one classical RK4 step (4 right-hand sides + stage combines) via
fr_rk4, replayed as a captured CUDA graph (the library's default); the metric
is N_V * sum_e N_e^(u) |Omega_e| * 4 * steps / time / 1e9.  Per-kernel times
come from a second pass over the same steps with kernel timing on (direct
launches, CUDA events around every kernel).  The comparison legs (FP64, FP32,
BF16x3) are timed per RK stage as well, and the error of each precision's
RHS against the FP64 GPU RHS of the same state is stated per variable.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RHS GDOF/s per RK stage (mixed vs plain FP64 GPU) and % of HBM/tensor roofline"
UNIT = "GDOF/s"
PRM = dict(gamma=1.4, mu=1.0 / 1600.0, prandtl=0.71, ldg_beta=0.5, ldg_tau=0.1)
# perturbation form about the Taylor-Green mean state (rho0 = 1, p0 = 1/(gamma M^2), M = 0.1)
REF = dict(ref_rho=1.0, ref_p=1.0 / (1.4 * 0.1 ** 2))


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=96, help="elements per box edge")
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "fp64", "bf16x3", "tf32x3"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison leg")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 CUDA-core comparison leg")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16x3 tensor-core comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed quad/triangle annulus leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (16^3 hex box) leg")
    ap.add_argument("--autotune", action="store_true",
                    help="autotune kernel variants missing from the committed table (outside the timed region)")
    ap.add_argument("--dense", action="store_true",
                    help="run the headline context with the dense operator products (tensor cores on the split "
                         "precisions) instead of the structured kernels: for profiling the dense path")
    ap.add_argument("--extra-legs", action="store_true",
                    help="also time the SD / HU correction functions and the Euler / DOPRI5 steppers (64^3 box)")
    return ap.parse_args()


# ---------------------------------------------------------------- CPU oracle leg
def _oracle_system(n_sample, order):
    from fr_inputs import periodic_box, fields
    from oracle.system import FRSystem
    m = periodic_box("hex", n_sample, 0.0, 2 * np.pi)
    o = FRSystem(m, order, "ns", **PRM)
    U = [fields.perturbed_taylor_green(o.solution_coords(0), M=0.1).transpose(1, 0, 2).copy()]
    return o, U


def _oracle_worker(n_sample, order, warmup, reps, barrier, queue):
    """One oracle process: set up, warm up, wait for the others, time `reps` RHS."""
    try:
        o, U = _oracle_system(n_sample, order)
        for _ in range(warmup):
            o.rhs(U)
        barrier.wait(timeout=900)
        t0 = time.perf_counter()
        for _ in range(reps):
            o.rhs(U)
        queue.put((U[0].size, reps, time.perf_counter() - t0))
    except Exception as e:                                    # reported, not hidden
        queue.put(("error", repr(e), 0.0))


def oracle_processes(n_sample, order, nproc, warmup, reps):
    """Time the FP64 oracle's RHS in `nproc` independent processes at once
    (spawned, one host thread each: numpy's einsum contractions are single-
    threaded and the thread pools are pinned to one thread), each on its own
    copy of the periodic n_sample^3 sample.  Returns (GDOF/s over all
    processes, slowest process's seconds per RHS, processes)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        barrier, queue = ctx.Barrier(nproc), ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker, args=(n_sample, order, warmup, reps, barrier, queue))
                 for _ in range(nproc)]
        for pr in procs:
            pr.start()
        res = [queue.get(timeout=1800) for _ in procs]
        for pr in procs:
            pr.join()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    bad = [r for r in res if r[0] == "error"]
    if bad:
        raise RuntimeError(f"oracle process failed: {bad[0][1]}")
    tmax = max(r[2] for r in res)
    return sum(r[0] * r[1] for r in res) / tmax / 1e9, tmax / reps, nproc


def host_cores():
    """Cores this process may run on, and how many oracle processes of
    `per_proc_gb` fit in the available host memory."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    return n, avail


def oracle_baseline(order, n_sample=16):
    """The oracle on the host cores: one process alone (the 1-thread figure),
    then one process per core at once (memory permitting), both on the
    periodic n_sample^3 sample of the workload."""
    n, avail = host_cores()
    per_proc = 1.2e9 * (n_sample / 16.0) ** 3             # measured peak RSS ~0.8 GB at 16^3, p=4
    nproc = max(1, min(n, int(0.7 * avail / per_proc) if avail else n))
    one, t_one, _ = oracle_processes(n_sample, order, 1, 1, 2)
    allc, t_all, used = oracle_processes(n_sample, order, nproc, 1, 2)
    dof = n_sample ** 3 * (order + 1) ** 3 * 5
    return dict(value=allc, unit=UNIT, cores=used, kind="oracle", host_cores=n,
                single_thread_value=one,
                sample=f"periodic {n_sample}^3 hexes, p={order}, NS, FP64 numpy oracle ({dof} DOF per copy); "
                       f"{used} independent processes (one thread each) ran 2 RHS each at once after one "
                       f"warm-up, {t_all:.2f} s per RHS in the slowest; alone: {t_one:.2f} s per RHS "
                       f"(single_thread_value); rated per DOF per RHS")


def workload_config(a, world):
    """The benchmark workload (both arms report it): the periodic n^3 hex box at
    order p, 3D NS (5 variables), (p+1)^3 solution points per element."""
    nelem = a.n ** 3
    dof = nelem * (a.order + 1) ** 3 * 5
    return dict(workload=f"3D Navier-Stokes Taylor-Green (+seeded perturbation), periodic {a.n}^3 hex box, "
                         f"p={a.order}, {dof} DOF, context precision {a.precision}"
                         + (" (dense operator products)" if getattr(a, "dense", False)
                            else " (operator products on the FP32 structured kernels of hexahedra)"),
                elements=nelem, order=a.order, dof=dof, step="one RK4 step (4 RHS + stage combines)",
                parallelism=f"replicas x{world}")


def run_reference(a):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores;
    each step is one oracle RHS in every process on its own bounded 8^3
    sample of the workload (same order, physics and state), rated per DOF."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n, avail = host_cores()
    nproc = max(1, min(n, int(0.7 * avail / 0.3e9) if avail else n))
    val, t_rhs, used = oracle_processes(8, a.order, nproc, a.warmup, a.steps)
    dof8 = 8 ** 3 * (a.order + 1) ** 3 * 5
    sample = (f"periodic 8^3 hexes, p={a.order}, NS, FP64 numpy oracle, {used} independent processes (one thread "
              f"each), {a.steps} RHS each after {a.warmup} warm-up; {dof8} DOF per copy")
    cfg = dict(workload_config(a, 1))
    cfg["workload"] = (f"FP64 CPU oracle on a bounded sample of the benchmark workload ({sample}); the workload: "
                       + cfg["workload"])
    line = dict(impl="reference", metric=METRIC, value=val, unit=UNIT, n_gpus=a.gpus, steps=a.steps,
                warmup=a.warmup, ms_per_step=t_rhs * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", config=cfg,
                cpu_baseline=dict(value=val, unit=UNIT, cores=used, kind="oracle", sample=sample),
                e2e=dict(value=val, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        # raw samples: FR_BENCH_CLOCKS_DIR if set (to keep them), else a temporary directory
        cdir = os.environ.get("FR_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(cdir, f"fr_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd.insert(1, f"--id={self.uuid}")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except OSError:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=mx, reasons=sorted(reasons),
                    samples=len(sm))


# ---------------------------------------------------------------- roofline bookkeeping
def kernel_work(name, nu, nf, V, D, nelem, npairs, s, fused=False, one_side=False, with_qf=False):
    """Algorithmic (bytes, flops) of one launch of each kernel on the whole block.

    Bytes count every value the kernel must read or write once (state, metric
    terms, per-pair tables); flops count the dense operator products as the
    paper defines them (App. A).  one_side: LDG beta = +-1/2, where one side of
    each pair has weight zero in the common solution and in the viscous common
    flux, so that side's U^(f) (common solution) or Q^(f) (common flux) is not
    read."""
    E = nelem
    if name == "disu_gemm":
        return (nu + nf) * V * s * E, 2.0 * nf * nu * V * E
    if name == "tgradu_gemm":
        # the gradient transform (gradcoru) runs in this kernel (tensor-core
        # epilogue or structured kernel): + metric terms adj(J) and 1/J, read once
        # per element; with_qf: the structured kernel also writes Q^(f) = M5 Q
        # (gradfpts), which then reads nothing more
        extra = (D * D * nu + nu) * s * E if fused else 0
        qf = (D * nf * V * s * E, 2.0 * D * nf * nu * V * E) if with_qf else (0, 0.0)
        return (nf + nu + D * nu) * V * s * E + extra + qf[0], 2.0 * D * nu * (nf + nu) * V * E + qf[1]
    if name == "gradfpts_gemm":
        return (nu + nf) * V * s * E, 2.0 * nf * nu * V * E
    if name == "tdivf_gemm":
        if fused:
            # RK4 stage combination in the epilogue: the stages read/write 3, 4, 4, 2
            # values per entry (u, acc, tmp) instead of writing R
            return ((nf + D * nu) * V + nu) * s * E + 13 * nu * V * s * E / 4, 2.0 * nu * (nf + D * nu) * V * E
        return ((nf + D * nu + nu) * V + nu) * s * E, 2.0 * nu * (nf + D * nu) * V * E
    if name == "gradcoru":
        return (2 * D * nu * V + D * D * nu + nu) * s * E, 0.0
    if name == "tdisf":
        return (nu * V + 2 * D * nu * V + D * D * nu) * s * E, 0.0
    if name == "comm_sol":
        return npairs * ((3 if one_side else 4) * V * s + 8), 0.0
    if name == "comm_flux":
        return npairs * ((4 * V + (1 if one_side else 2) * D * V + D + 2) * s + 8), 0.0
    if name == "rk_stage":
        return 17 * nu * V * s * E / 4, 0.0       # stages read/write 4, 5, 5, 3 values per entry
    return None, None


# source files that define each profiled kernel: a committed traffic figure is
# used only while these files are unchanged
KERNEL_SOURCES = {
    "tc": ("fr_tc.cu", "fr_tc.hpp"),
    "pointwise": ("fr_kernels.cu", "fr_dev.hpp"),
}


def kernel_sources(kernel):
    # on the hexahedral benchmark every operator product runs on a structured
    # kernel (fr_kernels.cu); the tensor-core GEMMs serve triangles
    return KERNEL_SOURCES["pointwise"]


def source_sha(files):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1312_1638_b300", "csrc")
    for fn in sorted(files):
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload_key):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current sources of that kernel; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        tab = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = tab.get(f"{workload_key}/{kernel}")
    if not ent or ent.get("source_sha") != source_sha(kernel_sources(kernel)):
        return None
    return ent.get("bytes_per_launch")


# ---------------------------------------------------------------- replicas
def replica_value(ms_local, units_per_rank, world, dist=None, device="cpu"):
    """Whole-job throughput of `world` independent replicas: every rank
    processed units_per_rank units; the job time is the slowest rank's.
    Returns (value in units per second / 1e9, max ms over ranks)."""
    ms = ms_local
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return units_per_rank * world / (ms / 1e3) / 1e9, ms


def structured_nonzeros(nu, nf, D, order, with_qf=False):
    """Multiply-adds per output column of the products that run on structured
    kernels on a hexahedral (tensor) mesh: M0 (p+1 per flux-point row, for U^(f)
    and the gradient at flux points), the corrected gradient [M6 | M4 - M6 M0]
    (p+1 solution points and 2 flux points per row, D nu rows; with_qf: plus the
    D M0 products it then forms) and the divergence [M3 | M1 - M3 M2] (per
    direction p+1 flux values and 2 common fluxes, nu rows)."""
    p1 = order + 1
    return {"disu_gemm": nf * p1, "gradfpts_gemm": nf * p1,
            "tgradu_gemm": D * nu * (p1 + 2) + (D * nf * p1 if with_qf else 0),
            "tdivf_gemm": nu * D * (p1 + 2)}


def operator_flops_per_rhs(nu, nf, V, D, nelem):
    """Dense operator flops of one NS right-hand side (App. A)."""
    f = 0.0
    for k, n in (("disu_gemm", 1), ("tgradu_gemm", 1), ("gradfpts_gemm", D), ("tdivf_gemm", 1)):
        f += n * kernel_work(k, nu, nf, V, D, nelem, 0, 4)[1]
    return f


# ---------------------------------------------------------------- GPU leg
def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    cpu_baseline = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu_baseline = oracle_baseline(a.order)          # spawned processes, before any CUDA call

    import torch
    from fr_inputs import periodic_box, fields
    from paper_1312_1638_b300 import build as _build
    _build.build()
    from paper_1312_1638_b300 import fr

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # FP32 / FP64 CUDA-core peaks from unit counts and the maximum SM clock:
    # 148 SMs x 128 FP32 lanes x 2 flop; FP64 at the B300 rate of 1.25 TFLOP/s nominal.
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    fp32_nominal = 148 * 128 * 2 * sm_max * 1e6 / 1e12
    try:
        fp32_peak, fp64_peak = fr.fma_peak(local)
        alu_src = "measured FMA probe (fr_fma_peak)"
    except fr.FRError:
        fp32_peak, fp64_peak = fp32_nominal, 1.25
        alu_src = "nominal unit counts x clock"
    alu_peaks = dict(fp32_tflops=round(fp32_peak, 2), fp64_tflops=round(fp64_peak, 3), source=alu_src,
                     fp32_nominal_tflops=round(fp32_nominal, 1), fp64_nominal_tflops=1.25)

    t_setup = time.perf_counter()
    mesh = periodic_box("hex", a.n, 0.0, 2 * np.pi)
    s = fr.Solver(mesh, a.order, "ns", a.precision, device=local, **PRM, **REF)
    L = s.layout(0)
    nu, nf, V, nelem, ld = L["nupts"], L["nfpts"], L["nvars"], L["nelem"], L["ld"]
    D = 3
    dof = nu * V * nelem
    X = torch.from_numpy(s.solution_points(0)).cuda()
    U0 = fields.perturbed_taylor_green(X, M=0.1)                     # [V, nu, nelem]
    del X
    dt_np = torch.float64 if a.precision == "fp64" else torch.float32
    u = torch.zeros((nu, V, ld), dtype=dt_np, device="cuda")
    u[:, :, :nelem] = U0.permute(1, 0, 2).to(dt_np)
    del U0
    u_init = u.clone()
    # kernel-variant choices measured on B300 (committed table; --autotune measures missing entries)
    if a.dense:
        for opt in ("structured_interp", "structured_grad", "structured_div"):
            s.set_option(opt, 0)
    tune_src, tune_text = s.apply_tuning([u] if a.autotune else None)
    t_setup = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream()
    dt = 1e-4

    # warm-up: the first call captures the RK4 step as a CUDA graph
    for _ in range(a.warmup):
        s.rk4([u], dt, 1, stream)
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    # headline: the product's default path, one captured RK4 step replayed per step
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(uuid) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(a.steps):
            s.rk4([u], dt, 1, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    stages = 4 * a.steps
    value, ms = replica_value(ms, dof * stages, world, dist, "cuda")
    assert s.sync_status() == fr.OK
    # kernel-level pass: the same steps launched directly, each kernel between a
    # pair of CUDA events on the launch stream (graph replay is off while timing)
    s.profile_enable(True)
    s.profile_read()
    evp0, evp1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evp0.record(stream)
    for _ in range(a.steps):
        s.rk4([u], dt, 1, stream)
    evp1.record(stream)
    torch.cuda.synchronize()
    ms_prof = evp0.elapsed_time(evp1)
    prof = s.profile_read()
    s.profile_enable(False)
    s.check_finite([u])
    finite_ok = s.sync_status() == fr.OK
    launches = sum(v[0] for v in prof.values())          # the same kernels the graph replays

    # roofline of the dominant kernel: the binding one of its HBM time and its
    # arithmetic time (tensor cores for the split-precision GEMMs, CUDA cores otherwise)
    npairs = nelem * nf // 2
    srz = 8 if a.precision == "fp64" else 4
    tc_path = a.precision in ("tf32x3", "bf16x3")
    bf16_peak = peaks.get("bf16_tflops", 1800.0)
    arith = {  # precision -> (peak TFLOP/s, executed / algorithmic flops, unit name, source)
        "tf32x3": (bf16_peak * 1.1 / 2.25, 3.0, "TF32 tensor",
                   "measured BF16 dense x nominal TF32/BF16 ratio (1.1/2.25)"),
        "bf16x3": (bf16_peak, 3.0, "BF16 tensor", "measured BF16 dense (cuBLAS burst)"),
        "fp32": (fp32_peak, 1.0, "FP32 CUDA core", alu_src),
        "fp64": (fp64_peak, 1.0, "FP64", alu_src),
    }[a.precision]

    one_side = PRM["ldg_beta"] in (0.5, -0.5)
    # products that run on a structured kernel on this workload (hexahedra): the
    # nonzeros they multiply per column (M0 rows: p+1; corrected-gradient rows:
    # p+1 solution points and 2 flux points), as FP32 (FP64) multiply-adds on
    # the CUDA cores whatever the precision
    with_qf = prof.get("gradfpts_gemm", (0, 0.0))[0] == 0      # Q^(f) formed by the gradient kernel
    structured = {} if a.dense else structured_nonzeros(nu, nf, D, a.order, with_qf)
    # transform / RK stage in the kernel (the structured kernels; the dense
    # products fuse them on the tensor-core paths only)
    fused_of = {} if a.dense else {"tgradu_gemm": True, "tdivf_gemm": True}

    def roof_of(name, launches, tms):
        kb, kf = kernel_work(name, nu, nf, V, D, nelem, npairs, srz, fused_of.get(name, tc_path), one_side,
                             with_qf and name == "tgradu_gemm")
        avg = tms / launches / 1e3
        t_hbm = kb / (hbm_peak * 1e9) if kb else 0.0
        t_alu = (kf * arith[1]) / (arith[0] * 1e12) if kf else 0.0
        r = dict(kernel=name, avg_launch_ms=tms / launches, algorithmic_bytes_per_launch=kb,
                 algorithmic_flops_per_launch=kf, hbm_frac=(kb / avg / 1e9) / hbm_peak if kb else None)
        if name in structured:
            kx = 2.0 * structured[name] * V * nelem
            pk = fp64_peak if a.precision == "fp64" else fp32_peak
            t_alu = kx / (pk * 1e12)
            r["executed_flops_per_launch"] = kx
            r["structured"] = "CUDA-core multiply-adds of the operator's nonzeros (structured kernel)"
            if t_alu > t_hbm:
                r.update(bound="alu", achieved=kx / avg / 1e12, peak=pk, unit="TFLOP/s", peak_source=alu_src)
            else:
                r.update(bound="hbm", achieved=kb / avg / 1e9, peak=hbm_peak, unit="GB/s",
                         peak_source=f"{peak_src} hbm_gbs")
        elif t_alu > t_hbm:
            bound = "tensor" if a.precision in ("tf32x3", "bf16x3") else "alu"
            r.update(bound=bound, achieved=kf * arith[1] / avg / 1e12, peak=arith[0], unit="TFLOP/s",
                     peak_source=arith[3], work_factor=arith[1],
                     note="achieved counts executed tensor/ALU flops = algorithmic operator flops x work_factor "
                          "(3 products per split-precision multiply)" if arith[1] != 1.0 else None)
        else:
            r.update(bound="hbm", achieved=kb / avg / 1e9, peak=hbm_peak, unit="GB/s",
                     peak_source=f"{peak_src} hbm_gbs")
        r["frac"] = r["achieved"] / r["peak"]
        r["timed"] = ("kernel-level pass of the same steps right after the headline (direct launches, CUDA "
                      "events per kernel on the launch stream)")
        return r

    top = max(prof.items(), key=lambda kv: kv[1][1])
    roof = roof_of(top[0], *top[1])
    wk = f"hex{a.n}_p{a.order}_ns_{a.precision}"
    roof["traffic"] = measured_traffic(top[0], wk)
    total_ms = sum(x[1] for x in prof.values())
    per_kernel = {}
    for k, v in prof.items():
        if not v[0]:
            continue
        d = dict(launches=v[0], ms=round(v[1], 3), share=round(v[1] / max(total_ms, 1e-9), 4))
        b, f = kernel_work(k, nu, nf, V, D, nelem, npairs, srz, fused_of.get(k, tc_path), one_side,
                           with_qf and k == "tgradu_gemm")
        if b:
            d["GB_s"] = round(b / (d["ms"] / d["launches"] / 1e3) / 1e9, 1)
            d["hbm_frac"] = round(d["GB_s"] / hbm_peak, 3)
        if f:
            d["TFLOP_s_algorithmic"] = round(f / (d["ms"] / d["launches"] / 1e3) / 1e12, 2)
        per_kernel[k] = d

    # end to end through the C ABI with host buffers: every step copies the state
    # in from pinned host memory, runs one RK4 step and copies it back (fr_rk4_host)
    e2e = None
    if not a.no_e2e:
        uh = u_init.cpu().pin_memory()
        s.rk4_host([uh], dt, 1, stream)                      # staging allocation and graph capture
        ne = max(3, min(a.steps, 5))
        t0 = time.perf_counter()
        for _ in range(ne):
            s.rk4_host([uh], dt, 1, stream)
        te = (time.perf_counter() - t0) / ne
        nbytes = uh.numel() * uh.element_size()
        e2e = dict(value=dof * 4 * world / te / 1e9, unit=UNIT, h2d_bytes_per_step=nbytes,
                   d2h_bytes_per_step=nbytes, ms_per_step=round(te * 1e3, 2),
                   note="fr_rk4_host: per step H2D of U from pinned memory, one RK4 step (graph replay), D2H of "
                        "U, host-synchronous; rated per RK stage like the headline")
        del uh

    # reference result for the error statements below: the FP64 GPU RHS of the
    # same (FP32-rounded) state; the FP64 path matches the oracle to 1e-13 of the
    # terms' magnitude in the parity tests
    r_main = torch.empty_like(u_init)
    s.rhs([u_init], [r_main], stream)
    s.close()
    del u
    torch.cuda.empty_cache()

    def rel_l2_vs(r, ref):
        x = r[:, :, :nelem].double()
        num = ((x - ref) ** 2).sum(dim=(0, 2)).sqrt()
        den = (ref ** 2).sum(dim=(0, 2)).sqrt()
        return [float(v) for v in (num / den).cpu()]

    # comparison legs on the same mesh and state, per RK stage like the headline
    def rk_leg(prec, warm, reps, graphs=True):
        sl = fr.Solver(mesh, a.order, "ns", prec, device=local, **PRM, **REF)
        sl.apply_tuning()
        sl.set_option("graphs", 1 if graphs else 0)
        dtp = torch.float64 if prec == "fp64" else torch.float32
        ul = u_init.to(dtp, copy=True)                      # a copy: the leg's RK4 steps advance it
        rl = torch.empty_like(ul)
        sl.rhs([ul], [rl], stream)                          # loads every kernel
        if warm:
            sl.rk4([ul], dt, warm, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sl.rk4([ul], dt, reps, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps
        st_l = sl.sync_status()
        sl.close()
        del ul
        fl = operator_flops_per_rhs(nu, nf, V, D, nelem)
        # on hexahedra every operator product runs on a structured kernel: FP32
        # (FP64) multiply-adds of the operators' nonzeros on the CUDA cores
        sn = structured_nonzeros(nu, nf, D, a.order, True)
        ex = 2.0 * V * nelem * (sn["disu_gemm"] + sn["tgradu_gemm"] + sn["tdivf_gemm"])
        pk, pname = (fp64_peak, "FP64 FMA (measured)") if prec == "fp64" else (fp32_peak, "FP32 FMA (measured)")
        out = dict(gdofs_per_rk_stage=4 * dof / (t / 1e3) / 1e9, ms_per_rk4_step=t, precision=prec,
                   graphs=graphs, operator_tflops_algorithmic=round(4 * fl / (t / 1e3) / 1e12, 2),
                   executed_tflops_whole_step=round(4 * ex / (t / 1e3) / 1e12, 3), alu_peak_tflops=round(pk, 2),
                   alu_peak=pname, alu_frac_whole_step=round(4 * ex / (t / 1e3) / 1e12 / pk, 4),
                   status="ok" if st_l == fr.OK else fr.STATUS_NAMES[st_l],
                   note="algorithmic: the dense operator flops of App. A over the whole RK4 step time; executed: "
                        "the structured kernels' multiply-adds (all on the CUDA cores), all kernels' time included")
        return out, rl

    fp64, parity, r64 = None, None, None
    if not a.no_fp64 and a.precision != "fp64":
        # one RK4 step of the FP64 path takes seconds: direct launches, one step timed
        fp64, r64 = rk_leg("fp64", 0, 1, graphs=False)
        r64 = r64[:, :, :nelem].clone()
        torch.cuda.empty_cache()
        parity = dict(reference="FP64 GPU RHS of the same FP32-rounded state (full 96^3 box, every element)",
                      variables=["rho", "rho u", "rho v", "rho w", "E"],
                      rel_l2_per_var={a.precision: rel_l2_vs(r_main, r64)})
    del r_main
    fp32 = bf16 = None
    if not a.no_fp32 and a.precision != "fp32":
        fp32, r32 = rk_leg("fp32", 1, 2)
        if parity is not None:
            parity["rel_l2_per_var"]["fp32"] = rel_l2_vs(r32, r64)
        del r32
    if not a.no_bf16 and a.precision != "bf16x3":
        bf16, rb = rk_leg("bf16x3", 1, 3)
        if parity is not None:
            parity["rel_l2_per_var"]["bf16x3"] = rel_l2_vs(rb, r64)
        del rb
    del r64
    torch.cuda.empty_cache()
    # mixed-mesh workload: 2D NS on the annulus (100k quads + 60k triangles, p = 4, Re 100, M 0.2)
    mixed = None
    if not a.no_mixed:
        from fr_inputs import annulus_mixed
        p_inf = 1.0 / (1.4 * 0.2 ** 2)
        mprm = dict(gamma=1.4, mu=0.01, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1, bc_rho=1.0, bc_v=(1.0, 0.0, 0.0),
                    bc_p=p_inf, outflow_p=p_inf, wall_cpTw=1.4 / 0.4 * p_inf, ref_rho=1.0, ref_p=p_inf)
        mm = annulus_mixed()
        mixed = dict(workload="2D NS annulus r in [0.5, 20], 100,000 quads (curved wall ring) + 60,000 triangles, "
                              "p=4, Re 100, M 0.2, free-stream state plus a seeded smooth perturbation")
        for prec, nrep in ((a.precision, 20), ("fp64", 3)):
            sm = fr.Solver(mm, 4, "ns", prec, device=local, **mprm)
            mixed[f"{prec}_kernel_variants"] = sm.apply_tuning()[0]
            dtp = torch.float64 if prec == "fp64" else torch.float32
            um, mdof = [], 0
            for b in range(len(mm.blocks)):
                X = sm.solution_points(b)
                Ub = fields.smooth_random(X, seed=3, amp=0.1, vel0=(1.0, 0.0), p0=p_inf).transpose(1, 0, 2)
                um.append(torch.from_numpy(sm.pack(b, Ub)).to(dtp).cuda())
                mdof += Ub.size
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            # dt well inside the viscous limit of the wall ring (h ~ 0.006, p = 4, mu = 0.01)
            sm.rk4(um, 2e-6, 1 if prec == "fp64" else 3, stream)
            e0.record(stream)
            sm.rk4(um, 2e-6, nrep, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            mixed[f"{prec}_gdofs_per_rk_stage"] = mdof * 4 * nrep / (e0.elapsed_time(e1) / 1e3) / 1e9
            mixed[f"{prec}_ms_per_rk4_step"] = e0.elapsed_time(e1) / nrep
            sm.check_finite(um)
            st_m = sm.sync_status()
            mixed[f"{prec}_status"] = "ok" if st_m == fr.OK else fr.STATUS_NAMES[st_m]
            mixed["dof"] = mdof
            sm.close()
            del um
            torch.cuda.empty_cache()
    # Taylor-Green workload at p = 3: 32^3 hex box (10.5 M DOF), split precision vs the FP64 GPU path
    tgv32 = None
    if not a.no_mixed:
        mt = periodic_box("hex", 32, 0.0, 2 * np.pi)
        tgv32 = dict(workload="3D NS Taylor-Green, periodic 32^3 hex box, p=3, Re 1600, M 0.1")
        for prec, nrep in (("bf16x3", 20), (a.precision, 20), ("fp64", 3)):
            st_ = fr.Solver(mt, 3, "ns", prec, device=local, **PRM, **REF)
            st_.apply_tuning()
            dtp = torch.float64 if prec == "fp64" else torch.float32
            Ut = fields.taylor_green(st_.solution_points(0), M=0.1)          # [V, nupts, nelem], host
            ut = torch.from_numpy(st_.pack(0, Ut.transpose(1, 0, 2))).to(dtp).cuda()
            tdof = Ut.size
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            st_.rk4([ut], 2e-4, 1 if prec == "fp64" else 3, stream)
            e0.record(stream)
            st_.rk4([ut], 2e-4, nrep, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            tgv32[f"{prec}_gdofs_per_rk_stage"] = tdof * 4 * nrep / (e0.elapsed_time(e1) / 1e3) / 1e9
            tgv32["dof"] = tdof
            st_.close()
            del ut, Ut
            torch.cuda.empty_cache()
    # adjoint workload: 16^3 hex box, p = 4, Taylor-Green + seeded perturbation (M 0.1); the adjoint RHS
    # against the forward RHS on the same state, and the adjoint of 50 RK4 steps (dt 1e-3, checkpoints
    # every 10), Euler and Navier-Stokes
    adjoint = None
    if not a.no_adjoint:
        ma = periodic_box("hex", 16, 0.0, 2 * np.pi)
        adjoint = dict(workload="periodic 16^3 hex box, p=4, Taylor-Green + seeded perturbation, M 0.1; "
                                "Euler and NS (Re 1600); adjoint of one RHS and of 50 RK4 steps (dt 1e-3, "
                                "checkpoints every 10, checkpoint allocation included)")
        rng_a = np.random.default_rng(4242)
        for sysname in ("euler", "ns"):
            for prec in ("fp32", a.precision):
                kw = dict(PRM, **REF) if sysname == "ns" else dict(gamma=1.4, **REF)
                sa = fr.Solver(ma, 4, sysname, prec, device=local, **kw)
                Ua = fields.perturbed_taylor_green(sa.solution_points(0), M=0.1).transpose(1, 0, 2)
                ua = torch.from_numpy(sa.pack(0, Ua)).float().cuda()
                la = torch.from_numpy(sa.pack(0, rng_a.standard_normal(Ua.shape))).float().cuda()
                ra, oa = torch.empty_like(ua), torch.empty_like(ua)
                sa.rhs([ua], [ra], stream)
                sa.adjoint_rhs([ua], [la], [oa], stream)
                torch.cuda.synchronize()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
                nrep = 20
                ev[0].record(stream)
                for _ in range(nrep):
                    sa.rhs([ua], [ra], stream)
                ev[1].record(stream)
                for _ in range(nrep):
                    sa.adjoint_rhs([ua], [la], [oa], stream)
                ev[2].record(stream)
                ev[3].record(stream)
                sa.rk4_adjoint([ua], [la], 1e-3, 50, 10, stream)
                ev[4].record(stream)
                torch.cuda.synchronize()
                t_f, t_a = ev[0].elapsed_time(ev[1]) / nrep, ev[1].elapsed_time(ev[2]) / nrep
                t_rk = ev[3].elapsed_time(ev[4])
                sa.check_finite([la])
                st_a = sa.sync_status()
                adjoint[f"{sysname}_{prec}"] = dict(
                    ms_rhs=round(t_f, 4), ms_adjoint_rhs=round(t_a, 4), adjoint_over_rhs=round(t_a / t_f, 2),
                    adjoint_gdofs=round(Ua.size / (t_a / 1e3) / 1e9, 2), ms_rk4_adjoint_50_steps=round(t_rk, 2),
                    status="ok" if st_a == fr.OK else fr.STATUS_NAMES[st_a])
                adjoint["dof"] = Ua.size
                sa.close()
                del ua, la, ra, oa
                torch.cuda.empty_cache()
    # rows without a leg of their own in the default run: the SD / HU correction functions (the DG
    # kernels with other operator values) and the forward Euler / DOPRI5 steppers, on a 64^3 box
    extra = None
    if a.extra_legs:
        mx = periodic_box("hex", 64, 0.0, 2 * np.pi)
        extra = dict(workload=f"periodic 64^3 hex box, p={a.order}, NS Taylor-Green + seeded perturbation, "
                              f"precision {a.precision}")
        dtx = torch.float64 if a.precision == "fp64" else torch.float32
        for corr in ("dg", "sd", "hu"):
            sx = fr.Solver(mx, a.order, "ns", a.precision, device=local, correction=corr, **PRM, **REF)
            Ux = fields.perturbed_taylor_green(sx.solution_points(0), M=0.1).transpose(1, 0, 2)
            ux = torch.from_numpy(sx.pack(0, Ux)).to(dtx).cuda()
            rx = torch.empty_like(ux)
            sx.rhs([ux], [rx], stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(10):
                sx.rhs([ux], [rx], stream)
            e1.record(stream)
            torch.cuda.synchronize()
            extra[f"{corr}_gdofs_per_rhs"] = round(Ux.size * 10 / (e0.elapsed_time(e1) / 1e3) / 1e9, 2)
            if corr == "dg":
                # 5 steps of each stepper after one warm-up step; DOPRI5 evaluates 7 RHS on a call's
                # first step and 6 on the others (first stage reused)
                n = 5
                for name, fn, nrhs in (("rk4", lambda k: sx.rk4([ux], 1e-4, k, stream), 4.0),
                                       ("euler", lambda k: sx.euler([ux], 1e-5, k, stream), 1.0),
                                       ("dopri5", lambda k: sx.dopri5([ux], 1e-4, k, stream=stream),
                                        (7.0 + 6.0 * (n - 1)) / n)):
                    fn(1)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    fn(n)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms_s = e0.elapsed_time(e1) / n
                    extra[f"{name}_ms_per_step"] = round(ms_s, 3)
                    extra[f"{name}_gdofs_per_rhs"] = round(Ux.size * nrhs / (ms_s / 1e3) / 1e9, 2)
            sx.check_finite([ux])
            stx = sx.sync_status()
            extra[f"{corr}_status"] = "ok" if stx == fr.OK else fr.STATUS_NAMES[stx]
            extra["dof"] = Ux.size
            sx.close()
            del ux, rx
            torch.cuda.empty_cache()

    if rank != 0:
        return 0
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=a.steps, warmup=a.warmup,
        ms_per_step=ms / a.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
        # the arithmetic the timed path computes in: on hexahedra every product runs
        # on the FP32 structured kernels whatever the context's precision; with
        # --dense the split-precision tensor-core products run
        dtype=("f64" if a.precision == "fp64" else
               {"fp32": "f32", "tf32x3": "tf32x3+f32", "bf16x3": "bf16x3+f32"}[a.precision] if a.dense else "f32"),
        data="synthetic",
        config=dict(workload_config(a, world),
                    l2="inputs larger than L2 (state alone is %.1f GB)" % (u_init.numel() * u_init.element_size() / 1e9),
                    setup_s=round(t_setup, 1), kernel_variants=dict(source=tune_src, choice=tune_text),
                    operator_products="dense (--dense)" if a.dense else "structured kernels on hexahedra"),
        roofline=roof, cpu_baseline=cpu_baseline, e2e=e2e, gpu_launches=launches,
        clocks=clk.summary(), per_kernel=per_kernel, kernel_pass_ms_per_step=ms_prof / a.steps,
        parity=parity, fp32_gpu=fp32, fp64_gpu=fp64, bf16x3_gpu=bf16, mixed_mesh=mixed, tgv32_p3=tgv32,
        adjoint_16cube_p4=adjoint, corrections_steppers_64cube=extra,
        alu_peaks=alu_peaks, finite=finite_ok,
    )
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
