#!/usr/bin/env python3
"""Benchmark of the matrix-free SIMP hot path on one GB300.

A step is one SIMP iteration of the 120 x 60 x 30 cantilever (216,000 Q1
elements, 686,433 DOFs; x=0 face clamped, unit -y load on the bottom edge of
the free end; V_f = 0.3, r_min = 1.5, E0 = 1, Emin = 1e-9, nu = 0.3, p = 3):
cone filter -> SIMP modulus -> Jacobi diagonal -> linear solve to
||f - Ku||/||f|| <= 1e-8 (warm start) -> compliance and sensitivities ->
filter transpose -> OC bisection.  Every step runs in the library's CUDA
kernels; the steps continue one SIMP run from the uniform start (the warm-up
steps are its first iterations).  The solve is the chosen form (--form
mixed, default: FP64 iterative refinement around an FP32 inner Jacobi-PCG)
or plain FP64 Jacobi-PCG (--form f64); with the mixed form the same steps
are also run with plain FP64 from the same state ("plain_fp64": its SIMP
iteration time and the largest relative compliance difference), and with the
multigrid solver ("gmg": V-cycle CG in FP64 refinement, its SIMP iteration
time and speed-ups).

value: K.v throughput of the whole step, n_elem x (K.v applications in the
timed steps) / (device time of the timed steps), in Gelem/s, with inputs
resident in HBM and L2 flushed (256 MiB write) before every step.
e2e: the same through the public API from pinned host buffers, the per-step
host->device copy of rho, u, f and the device->host copy of rho, u inside
the timed region.  roofline: the dominant kernel (the K.v of the PCG), its
average launch duration from CUDA events around a graph of 64 back-to-back
launches of the same kernel, grid and arguments (mfto_cg_kv_time), beside
the duration from CUDA events recorded around every launch in a replay of
the same steps (which adds two event nodes to each launch).  cpu_baseline:
the CPU oracle on a bounded sample of the same step (its PCG capped),
single-threaded, plus an all-cores sample of its K.v.

--impl reference times the CPU oracle alone (the method's plain restatement)
on the same workload and metric.
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
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "K·v Gelem/s & % roofline; SIMP iter time, plain FP64 vs chosen forms @1e-6"
WORKLOAD = "cantilever_120x60x30"
FLOP_PER_ELEM = 1152.0                       # 2 * 24 * 24, dense element contraction
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
IR_MODES = {"restart": 0, "continue": 1}
# DRAM bytes (read + write) per launch of the dominant kernels from one ncu
# capture (profiles/kv_f32_cg2_cantilever_120x60x30_full.md,
# profiles/kv_f32_cg2_cantilever_256x128x150_full.md,
# profiles/kv_f64_pcg_cantilever_256x128x150_full.md, the FP64 figure scaled from
# 4,915,200 to 216,000 elements by the bytes it reads per element), cold caches,
# each with a digest of the kernel's source files at capture time: when the
# sources change the figure is reported as stale (null) until it is re-taken.
KERNEL_SOURCES = {
    "cg2_kv_kernel": ["kv_column.cuh", "pcg_f32.cu", "modes.cuh"],
    "pcg_kv_tile_kernel<double>": ["kv_tile.cuh", "kv_tile.cu", "modes.cuh"],
}
NCU_DRAM_BYTES = {
    ("cg2_kv_kernel<2>", WORKLOAD): (6.646272e6, "0c045bd0c8e8"),
    ("cg2_kv_kernel<3>", WORKLOAD): (6.649088e6, "0c045bd0c8e8"),
    ("cg2_kv_kernel<2>", "cantilever_256x128x150"): (143.325184e6 + 74.990592e6, "0c045bd0c8e8"),
    ("cg2_kv_kernel<3>", "cantilever_256x128x150"): (144.233472e6 + 74.192384e6, "0c045bd0c8e8"),
    ("pcg_kv_tile_kernel<double>", WORKLOAD): ((293.127936e6 + 199.873024e6) * 216000 / 4915200,
                                               "6e176c6f4f1e"),
}


def source_digest(kernel: str) -> str:
    import hashlib
    base = kernel.split("<")[0] if kernel.startswith("cg2_") else kernel
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(base, []):
        h.update((ROOT / "paper_2604_18020_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:12]


def ncu_traffic(kernel: str, workload: str):
    """(bytes, note): the captured DRAM bytes per launch, or None when there is
    no capture or the kernel's sources changed since it was taken."""
    rec = NCU_DRAM_BYTES.get((kernel, workload))
    if rec is None:
        return None, "no ncu capture of this kernel and workload"
    if source_digest(kernel) != rec[1]:
        return None, "stale: the kernel's sources changed since the ncu capture"
    return rec[0], "ncu dram__bytes_read.sum + dram__bytes_write.sum, one cold launch"


REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def measured_hbm_gbs():
    try:
        return float(json.loads((ROOT / "MEASURED_PEAKS.json").read_text())["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0          # the profiling recipe's fallback figure


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="mfto_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={SMI_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        lines = []
        if self.path and os.path.exists(self.path):
            with open(self.path) as fh:
                lines = fh.readlines()
            os.unlink(self.path)
        return clock_summary(lines)


def clock_summary(lines):
    """Median SM clock, the largest max-clock reading and the throttle
    reasons seen active, from nvidia-smi CSV rows of SMI_FIELDS (no header,
    no units); malformed rows are skipped."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
        except ValueError:
            continue
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    reasons = sorted({REASONS[i] for _, _, flags in rows for i, f in enumerate(flags)
                      if f.lower() == "active"})
    return {"sm_mhz": statistics.median(r[0] for r in rows),
            "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
            "samples": len(rows)}


def reduce_over_ranks(dist, device, maxes, sums):
    """The benchmark's reduction over ranks: the largest of each timing in
    `maxes` and the total of each count in `sums` (the ranks are independent
    replicas; besides this and the barriers around the timed region they
    exchange nothing).  dist = None (one process) returns both lists
    unchanged."""
    maxes, sums = [float(x) for x in maxes], [float(x) for x in sums]
    if dist is None:
        return maxes, sums
    import torch
    tm = torch.tensor(maxes, dtype=torch.float64, device=device)
    ts = torch.tensor(sums, dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    return tm.tolist(), ts.tolist()


# ------------------------------------------------------------ CPU oracle leg

def oracle_step(P, rho, u, maxit, rtol=1e-8):
    """One SIMP iteration of the CPU oracle with the PCG capped at maxit;
    returns (rho_new, u, kv_applications)."""
    import numpy as np
    from oracle import fem, filter as cone, simp, solve
    m = P.mesh
    KE = fem.ke_exact(1.0, 0.3)
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fixed = fem.dof_mask(P.fixed)
    count = [0]

    def apply_K(v):
        count[0] += 1
        return fem.kv(KE, E, edof, v, fixed)

    rho_phys = cone.filter_fwd(rho, m.nelx, m.nely, m.nelz, P.rmin)
    E = fem.simp_modulus(rho_phys, 3.0)
    d = fem.jacobi_diag(KE, E, edof, fixed)
    u, _ = solve.pcg(apply_K, d, P.f, u, rtol, maxit)
    _, dc_phys = simp.compliance_sens(KE, edof, u, rho_phys, 3.0)
    dc = cone.filter_T(dc_phys, m.nelx, m.nely, m.nelz, P.rmin)
    rho_new, _ = simp.oc_update(rho, dc, P.volfrac, 0.2)
    return rho_new, u, count[0]


def cpu_sample(workload: str, steps: int, maxit: int):
    import numpy as np
    from paper_2604_18020_gb300 import workloads as W
    P = W.WORKLOADS[workload]()
    rho = np.full(P.mesh.n_elem, P.volfrac)
    u = np.zeros(P.mesh.n_dof)
    times, kvs = [], []
    for _ in range(steps):
        t = time.perf_counter()
        rho, u, n = oracle_step(P, rho, u, maxit)
        times.append(time.perf_counter() - t)
        kvs.append(n)
    return {"times": times, "kv": kvs, "n_elem": P.mesh.n_elem}


# All-cores timing of the oracle's K.v: node slabs along z, one per worker
# process (spawned, no CUDA); each worker applies the oracle's element loop to
# the elements touching its slab and writes only its own nodes' rows, so the
# slabs need no reduction (race-free node ownership).
_MP = {}


def _mp_init(workload, v_name, y_name):
    import numpy as np
    from multiprocessing import shared_memory
    from oracle import fem
    from paper_2604_18020_gb300 import workloads as W
    P = W.WORKLOADS[workload]()
    m = P.mesh
    sv = shared_memory.SharedMemory(name=v_name)
    sy = shared_memory.SharedMemory(name=y_name)
    _MP.update(m=m, KE=fem.ke_exact(1.0, 0.3), edof=fem.edof_table_fast(m.nelx, m.nely, m.nelz),
               fd=fem.dof_mask(P.fixed),
               E=fem.simp_modulus(W.rho_random(m, seed=1), 3.0),
               v=np.ndarray((m.n_dof,), dtype=np.float64, buffer=sv.buf),
               y=np.ndarray((m.n_dof,), dtype=np.float64, buffer=sy.buf), shm=(sv, sy))


def _mp_slab(k_range):
    import numpy as np
    from oracle import fem
    k0, k1 = k_range
    m, edof, fd, v, y = _MP["m"], _MP["edof"], _MP["fd"], _MP["v"], _MP["y"]
    per_layer = m.nelx * m.nely
    kl, kh = max(k0 - 1, 0), min(k1, m.nelz)           # element layers touching the slab
    e0, e1 = kl * per_layer, kh * per_layer
    dpl = 3 * (m.nelx + 1) * (m.nely + 1)              # DOFs per node layer
    b0, b1 = kl * dpl, (kh + 1) * dpl                  # the DOFs those elements reach
    pv = np.where(fd[b0:b1], 0.0, v[b0:b1])
    w = fem.kv_unmasked(_MP["KE"], _MP["E"][e0:e1], edof[e0:e1] - b0, pv)
    d0, d1 = k0 * dpl, k1 * dpl
    y[d0:d1] = np.where(fd[d0:d1], v[d0:d1], w[d0 - b0:d1 - b0])
    return k1 - k0


def cpu_allcores_kv(workload: str, reps: int = 10):
    """The oracle's K.v on all host cores (one worker process per core, node
    slabs), checked against the single-process oracle; Gelem/s."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import numpy as np
    from oracle import fem
    from paper_2604_18020_gb300 import workloads as W
    P = W.WORKLOADS[workload]()
    m = P.mesh
    ncore = os.cpu_count() or 1
    sv = shared_memory.SharedMemory(create=True, size=8 * m.n_dof)
    sy = shared_memory.SharedMemory(create=True, size=8 * m.n_dof)
    try:
        v = np.ndarray((m.n_dof,), dtype=np.float64, buffer=sv.buf)
        y = np.ndarray((m.n_dof,), dtype=np.float64, buffer=sy.buf)
        v[:] = W.vec_random(m.n_dof, seed=1)
        nz = m.nelz + 1
        bounds = np.linspace(0, nz, min(ncore, nz) + 1).astype(int)
        slabs = [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        ctx = mp.get_context("spawn")
        with ctx.Pool(len(slabs), initializer=_mp_init, initargs=(workload, sv.name, sy.name)) as pool:
            pool.map(_mp_slab, slabs)                      # warm-up
            t = time.perf_counter()
            for _ in range(reps):
                pool.map(_mp_slab, slabs)
            dt = (time.perf_counter() - t) / reps
        ref = fem.kv(fem.ke_exact(1.0, 0.3), fem.simp_modulus(W.rho_random(m, seed=1), 3.0),
                     fem.edof_table_fast(m.nelx, m.nely, m.nelz), np.array(v),
                     fem.dof_mask(P.fixed))
        err = float(np.abs(y - ref).max() / np.abs(ref).max())
        if err > 1e-13:
            raise RuntimeError(f"all-cores oracle K.v differs from the oracle by {err:.2e}")
        return {"value": m.n_elem / dt / 1e9, "unit": "Gelem/s", "cores": len(slabs),
                "kv_s": dt, "max_rel_diff_vs_single": err}
    finally:
        sv.close(); sv.unlink()
        sy.close(); sy.unlink()


def cpu_simp_cfg0(n_iter: int = 20):
    """Uncapped SIMP iterations of the 24 x 12 x 12 cantilever by the oracle
    (PCG to rtol 1e-8), single-threaded; wall time per SIMP iteration."""
    from oracle import simp
    from paper_2604_18020_gb300 import workloads as W
    P = W.WORKLOADS["cantilever_24x12x12"]()
    m = P.mesh
    t = time.perf_counter()
    _, _, hist = simp.simp(m.nelx, m.nely, m.nelz, P.f, P.fixed, P.volfrac, P.rmin, n_iter)
    dt = time.perf_counter() - t
    return {"workload": "cantilever_24x12x12", "iterations": n_iter, "wall_s": dt,
            "s_per_iteration": dt / n_iter, "cg_iterations": int(sum(hist.cg_iterations)),
            "final_compliance": hist.compliance[-1], "threads": 1}


def run_cpu_sample(workload, steps, maxit, extra=False):
    """The oracle in a fresh process (spawned, no CUDA), one BLAS thread per
    process; extra: also the all-cores K.v and the uncapped 24 x 12 x 12 SIMP
    iterations."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--cpu-sample", workload,
                          "--steps", str(steps), "--maxit", str(maxit)]
                         + (["--cpu-extra"] if extra else []),
                         capture_output=True, text=True, env=env, cwd=str(ROOT))
    if out.returncode != 0:
        raise RuntimeError(f"CPU oracle sample failed:\n{out.stderr[-2000:]}")
    return json.loads(out.stdout.strip().splitlines()[-1])


def host_cpu():
    """The host's logical core count and CPU model name (from lscpu, else
    /proc/cpuinfo, else the machine type)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return os.cpu_count(), model or platform.machine()


def cpu_baseline_entry(res, maxit):
    tot_t = sum(res["times"])
    tot_kv = sum(res["kv"])
    n_cores, model = host_cpu()
    out = {"value": res["n_elem"] * tot_kv / tot_t / 1e9, "unit": "Gelem/s", "cores": 1,
           "host_cores": n_cores, "cpu_model": model,
           "kind": "oracle",
           "sample": f"{len(res['times'])} SIMP iteration(s) of {WORKLOAD} by the FP64 numpy "
                     f"oracle from the uniform start, PCG capped at {maxit} iterations "
                     f"({tot_kv} K.v applications, {tot_t:.1f} s, 1 BLAS thread)"}
    if "all_cores" in res:
        out["all_cores_kv"] = dict(res["all_cores"], sample=(
            f"the oracle's K.v on {WORKLOAD}, one spawned process per core over node slabs "
            f"along z (race-free: each process writes its own nodes), 10 applications"))
    if "simp_cfg0" in res:
        out["simp_cfg0_uncapped"] = res["simp_cfg0"]
    return out


# ------------------------------------------------------------- GPU leg

def cg_kv_roofline(m, kv_avg_s, sm_mhz, n_sm):
    """Roofline of one launch of the FP32 CG K.v on mesh m: algorithmic
    bytes (reads z, p_old, E, the node mask; writes p_new, q) and the dense
    element contraction (1152 flop per element) against the measured HBM
    copy bandwidth and the FP32 FMA pipe at the sampled SM clock; the slower
    of the two is the bound."""
    bytes_per_launch = m.n_node * (4 * 12 + 1) + 4 * m.n_elem
    hbm = measured_hbm_gbs()
    fp32_peak_tflops = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    t_bytes = bytes_per_launch / (hbm * 1e9)
    t_flops = FLOP_PER_ELEM * m.n_elem / (fp32_peak_tflops * 1e12)
    out = {"bytes_per_launch": bytes_per_launch, "flop_per_elem": FLOP_PER_ELEM,
           "frac_hbm": t_bytes / kv_avg_s, "frac_fp32_pipe": t_flops / kv_avg_s}
    if t_bytes >= t_flops:
        out.update({"bound": "hbm", "achieved": bytes_per_launch / kv_avg_s / 1e9, "peak": hbm,
                    "unit": "GB/s",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy benchmark), of measured"})
    else:
        out.update({"bound": "alu", "achieved": FLOP_PER_ELEM * m.n_elem / kv_avg_s / 1e12,
                    "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                    "peak_source": f"FP32 FMA pipe, {n_sm} SMs x 128 FMA/clk x 2 flop x "
                                   f"{sm_mhz:.0f} MHz median SM clock under load"})
    out["frac"] = out["achieved"] / out["peak"]
    return out


def large_kv_leg(dev, sm_mhz, n_sm, iters=400, workload="cantilever_256x128x150", shape=None,
                 engine=2):
    """The FP32 CG K.v on the 256 x 128 x 150 cantilever (4,915,200 elements,
    15.0M DOFs; another workload if given): one mixed solve of a filtered
    random design from u = 0, its inner CG capped at `iters` iterations (one
    refinement step), the launch shape autotuned, CUDA events around every
    K.v launch."""
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W
    P = W.WORKLOADS[workload]()
    m = P.mesh
    h = mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                    params=mfto.default_params(volfrac=P.volfrac, rmin=P.rmin, rtol=1e-8))
    try:
        h.set_cg_engine(engine)
        if shape:
            h.set_kv_shape(*shape)
            tuned = (shape[0], shape[1], None)
        else:
            tuned = h.kv_autotune()
        h.set_solver(mfto.FORM_F32, 1e-8, iters, 1)
        h.set_ir_mode(IR_MODES["continue"])
        rho = torch.tensor(W.rho_binary(m, seed=2, volfrac=P.volfrac), device=dev)
        rho_phys = torch.empty_like(rho)
        h.filter(rho, rho_phys)
        E = torch.empty_like(rho)
        h.simp_modulus(rho_phys, E)
        f = torch.tensor(P.f, device=dev)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
        h.ir_solve(E, f, u, inner_tol=1e-8)          # warm-up: graph capture
        u.zero_()
        h.kv_timing(True)
        st = h.ir_solve(E, f, u, inner_tol=1e-8)
        n, ms = h.kv_timing_read(mfto.FORM_F32)
        h.kv_timing(False)
        burst_us = h.cg_kv_time(16, 5) if engine == 2 else None
    finally:
        h.close()
    kv_events_s = ms * 1e-3 / max(n, 1)
    kv_avg_s = burst_us * 1e-6 if burst_us else kv_events_s
    roof = cg_kv_roofline(m, kv_avg_s, sm_mhz, n_sm)
    kname = (f"{'cg2_kv_kernel' if engine == 2 else 'pcg_kv_col_kernel'}"
             f"<{2 if tuned[1] == 0 else 3}>")
    tb, tnote = ncu_traffic(kname, workload)
    roof.update({"traffic": tb, "traffic_note": tnote})
    roof.update({"workload": workload, "elements": m.n_elem,
                 "kernel": (f"{'cg2_kv_kernel' if engine == 2 else 'pcg_kv_col_kernel'}"
                            f"<{2 if tuned[1] == 0 else 3}>"),
                 "kv_f32_zchunk": tuned[0], "kv_f32_kernel_kind": tuned[1],
                 "launches_timed": n, "kv_kernel_us": kv_avg_s * 1e6,
                 "kv_kernel_gelem_s": m.n_elem / kv_avg_s / 1e9,
                 "kv_kernel_us_timing": ("graph of 16 back-to-back launches, 5 timed replays "
                                         "(mfto_cg_kv_time)" if burst_us else
                                         "CUDA events around every launch in the CG graph"),
                 "kv_kernel_us_events_in_cg": kv_events_s * 1e6,
                 "inner_iterations": st.inner_iterations})
    return roof

def gpu_bench(args, rank, local_rank, world):
    import numpy as np
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    P = W.WORKLOADS[WORKLOAD]()
    m = P.mesh
    params = mfto.default_params(volfrac=P.volfrac, rmin=P.rmin, rtol=1e-8)
    h = mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed, params=params)
    tuned = None
    if args.form == "mixed":
        h.set_solver(mfto.FORMS[args.inner_form], args.inner_tol)
        h.set_cg_engine(args.cg_engine)
        h.set_ir_mode(IR_MODES[args.ir_mode])
        if args.kv_shape:
            # a pinned launch shape: profiling runs reproduce the shape the
            # autotuner picks in a plain run (its timings are distorted under a
            # profiler that serialises launches)
            nzc, kind = (int(x) for x in args.kv_shape.split(","))
            h.set_kv_shape(nzc, kind)
            tuned = (nzc, kind, None)
        elif not args.no_autotune:
            tuned = h.kv_autotune()
    rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=dev)
    u = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
    f = torch.tensor(P.f, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        h.simp_step(rho, u, f)
    torch.cuda.synchronize()
    rho0, u0 = rho.clone(), u.clone()

    def timed_pass(kv_timed: bool):
        rho.copy_(rho0)
        u.copy_(u0)
        h.kv_timing(kv_timed)
        total_ms, stats = 0.0, []
        l0 = h.launch_count()
        for _ in range(args.steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = h.simp_step(rho, u, f)
            b.record(stream)
            b.synchronize()
            total_ms += a.elapsed_time(b)
            stats.append(st)
        launches = h.launch_count() - l0
        kv64 = h.kv_timing_read(mfto.FORM_F64)
        kv32 = h.kv_timing_read(mfto.FORM_F32)
        cgt = h.cg_timing_read()
        h.kv_timing(False)
        return total_ms, stats, launches, kv64, kv32, cgt

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clocks:
        t_ms, stats, launches, _, _, _ = timed_pass(False)
    torch.cuda.synchronize()
    clk = clocks.summary()
    # replay with events around every K.v launch (same steps, same state)
    _, stats_b, _, kv64, kv32, cgt = timed_pass(True)
    cg = [s.cg_iterations for s in stats]
    assert cg == [s.cg_iterations for s in stats_b], "replay diverged"
    # K.v applications: FP64 launches, FP32 launches of the graph engine, and
    # the iterations of the persistent CG launches (one K.v each)
    kv_per_pass = kv64[0] + kv32[0] + cgt[1]
    persistent = args.form == "mixed" and cgt[0] > 0
    if persistent:
        kv_n, kv_ms = cgt[1], cgt[2]      # per CG iteration of the persistent kernel
    else:
        kv_n, kv_ms = kv32 if args.form == "mixed" else kv64   # the dominant K.v launches

    # e2e: public API from pinned host buffers, copies inside the timed region
    h_rho = rho0.cpu().pin_memory()
    h_u = u0.cpu().pin_memory()
    h_f = f.cpu().pin_memory()
    o_rho = torch.empty_like(h_rho).pin_memory()
    o_u = torch.empty_like(h_u).pin_memory()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rho.copy_(h_rho, non_blocking=True)
        u.copy_(h_u, non_blocking=True)
        f.copy_(h_f, non_blocking=True)
        h.simp_step(rho, u, f)
        o_rho.copy_(rho, non_blocking=True)
        o_u.copy_(u, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
        h_rho.copy_(o_rho)
        h_u.copy_(o_u)
    # plain FP64 Jacobi-PCG over the same steps from the same state, for the
    # "plain FP64 vs chosen form" comparison (skipped when the bench is FP64)
    fp64 = gmg_leg = None
    if args.form != "f64":
        h.set_solver(mfto.FORM_F64)
        t64, stats64, _, _, _, _ = timed_pass(False)
        c64 = [s.compliance for s in stats64]
        cf = [s.compliance for s in stats]
        fp64 = {"simp_iter_ms": t64 / args.steps,
                "cg_iterations": [s.cg_iterations for s in stats64],
                "compliance": c64,
                "max_compliance_rel_err": max(abs(a - b) / abs(b) for a, b in zip(cf, c64)),
                "speedup_of_chosen_form": t64 / t_ms}
        h.set_solver(mfto.FORMS[args.inner_form], args.inner_tol)
        # the same steps with the multigrid solver (V-cycle CG in FP64
        # refinement): the library's fastest SIMP iteration, beside the K.v one
        h.set_gmg_solver(True)
        h.simp_step(rho, u, f)            # warm-up: hierarchy storage, graph captures
        tg, statsg, _, _, _, _ = timed_pass(False)
        h.set_gmg_solver(False)
        cg_ = [s.compliance for s in statsg]
        gmg_leg = {"simp_iter_ms": tg / args.steps,
                   "solver_iterations": [s.cg_iterations for s in statsg],
                   "max_compliance_rel_err_vs_fp64": max(abs(a - b) / abs(b)
                                                         for a, b in zip(cg_, c64)),
                   "speedup_vs_plain_fp64": t64 / tg, "speedup_vs_chosen_form": t_ms / tg}
    # memory snapshot (the paper's VRAM table): the library's own device memory
    # (workspace and, after the multigrid leg, its hierarchy), PyTorch's peak
    # and the whole device's use
    free_b, total_b = torch.cuda.mem_get_info(dev)
    vram = {"library_bytes": h.device_bytes(),
            "torch_max_allocated_bytes": int(torch.cuda.max_memory_allocated(dev)),
            "device_used_bytes": int(total_b - free_b)}
    h2d = (h_rho.numel() + h_u.numel() + h_f.numel()) * 8
    d2h = (o_rho.numel() + o_u.numel()) * 8
    # the slowest rank's times and the K.v element applications of all ranks
    (t_ms, e2e_ms), (units,) = reduce_over_ranks(dist, dev, [t_ms, e2e_ms],
                                                 [m.n_elem * kv_per_pass])
    value = units / (t_ms * 1e-3) / 1e9
    e2e_value = units / (e2e_ms * 1e-3) / 1e9
    # the dominant kernel's duration: CUDA events around every K.v launch of
    # the replayed steps add the cost of two event nodes to each launch, so
    # the graph engine's K.v is also timed as a burst of back-to-back launches
    # of the same kernel, grid and arguments (mfto_cg_kv_time; after every
    # other leg, since it overwrites the FP32 work vectors)
    kv_events_s = kv_ms * 1e-3 / max(kv_n, 1)
    burst_us = burst_ev_us = None
    if (args.form == "mixed" and args.inner_form == "f32" and args.cg_engine == 2
            and not persistent):
        burst_us = h.cg_kv_time(64, 5)
        # the same burst with an event pair around every launch: what the
        # event nodes of the per-launch timing add to identical launches
        burst_ev_us = h.cg_kv_time(64, 5, events=True)
    kv_avg_s = burst_us * 1e-6 if burst_us else kv_events_s
    sm_mhz = clk["sm_mhz"] or 1950.0
    n_sm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    if args.form == "mixed":
        kname = ("pcg_kv_tile_kernel<float>" if args.inner_form == "f32"
                 else f"pcg_kv_tc_kernel ({args.inner_form})")
        if args.inner_form == "f32" and not persistent:
            kbase = "cg2_kv_kernel" if args.cg_engine == 2 else "pcg_kv_col_kernel"
            kname = f"{kbase}<{2 if tuned is None or tuned[1] == 0 else 3}>"
        roof = cg_kv_roofline(m, kv_avg_s, sm_mhz, n_sm)
        if persistent:
            # one CG iteration of the persistent kernel: the K.v phase plus the
            # vector update (reads u, p, q, r, 1/d; writes u, r, z: 32 B/DOF);
            # its time includes both grid barriers
            kname = "pcg_persist_f32 (per CG iteration: K.v + vector update + 2 grid barriers)"
            roof = cg_kv_roofline(m, kv_avg_s, sm_mhz, n_sm)
            roof["bytes_per_launch"] += 32 * m.n_dof
            roof["frac_hbm"] = roof["bytes_per_launch"] / (measured_hbm_gbs() * 1e9) / kv_avg_s
        tb, tnote = ncu_traffic(kname, WORKLOAD)
        roof.update({"traffic": tb, "traffic_note": tnote, "kernel": kname,
                     "duration_us": kv_avg_s * 1e6,
                     "duration_timing": ("graph of 64 back-to-back launches of the CG K.v, "
                                         "5 timed replays (mfto_cg_kv_time)" if burst_us else
                                         "CUDA events around every launch in the CG graph"),
                     "duration_us_events_in_cg": kv_events_s * 1e6,
                     "duration_us_burst_with_event_nodes": burst_ev_us if burst_us else None})
        if persistent:
            roof.update({"unit_of_work": "one CG iteration (one K.v application)",
                         "launches": cgt[0], "iterations_per_launch": cgt[1] / cgt[0],
                         "launch_us": cgt[2] * 1e3 / cgt[0]})
    else:
        fp64_peak_tflops = n_sm * 2 * 2 * sm_mhz * 1e6 / 1e12   # 2 DFMA/clk/SM, measured clock
        roof = {"bound": "alu", "achieved": FLOP_PER_ELEM * m.n_elem / kv_avg_s / 1e12,
                "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "kernel": "pcg_kv_tile_kernel<double>",
                "traffic": ncu_traffic("pcg_kv_tile_kernel<double>", WORKLOAD)[0],
                "peak_source": f"FP64 FMA pipe, {n_sm} SMs x 2 DFMA/clk x 2 flop x "
                               f"{sm_mhz:.0f} MHz median SM clock under load",
                "flop_per_elem": FLOP_PER_ELEM}
    roof["frac"] = roof["achieved"] / roof["peak"]
    large = None
    if args.form == "mixed" and args.inner_form == "f32" and not args.no_large and rank == 0:
        large = large_kv_leg(dev, sm_mhz, n_sm, engine=args.cg_engine)
    out = {
        "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.form == "f64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "elements": m.n_elem, "dofs": m.n_dof,
                   "form": args.form, "pcg_rtol": 1e-8,
                   "inner_tol": args.inner_tol if args.form == "mixed" else None,
                   "inner_form": args.inner_form if args.form == "mixed" else None,
                   "kv_kernel": roof.get("kernel"),
                   "cg_engine": ({0: "graph, last-block tickets", 1: "persistent",
                                  2: "graph, ticket-free"}[args.cg_engine]
                                 if args.form == "mixed" else "graph"),
                   "kv_f32_zchunk": tuned[0] if tuned else None,
                   "kv_f32_kernel_kind": tuned[1] if tuned else None,
                   "ir_mode": args.ir_mode if args.form == "mixed" else None,
                   "l2": "flushed before every step (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "simp_iter_ms": t_ms / args.steps,
        "cg_iterations": cg,
        "compliance": [s.compliance for s in stats],
        "kv_per_step": kv_per_pass / args.steps,
        "kv_f64_per_step": kv64[0] / args.steps,
        "kv_f32_per_step": kv32[0] / args.steps,
        "kv_kernel_us": kv_avg_s * 1e6,
        "kv_kernel_us_events_in_cg": kv_events_s * 1e6,
        "kv_kernel_gelem_s": m.n_elem / kv_avg_s / 1e9,
        "kv_f64_kernel_us": kv64[1] * 1e3 / max(kv64[0], 1),
        "roofline": roof,
        "kv_large": large,
        "e2e": {"value": e2e_value, "unit": "Gelem/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "plain_fp64": fp64,
        "gmg": gmg_leg,
        "vram": vram,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                   "reasons": clk["reasons"]},
    }
    h.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


def profile_run(args):
    """Short runs for ncu: 'profile' = W + K SIMP steps of the benchmark
    workload, nothing else; 'pcg' = one PCG capped at --maxit iterations on
    --workload with a seeded random density (exercises the CG K.v kernel on
    a mesh larger than L2)."""
    import numpy as np
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W
    dev = torch.device("cuda:0")
    P = W.WORKLOADS[args.workload]()
    m = P.mesh
    params = mfto.default_params(volfrac=P.volfrac, rmin=P.rmin, rtol=1e-8,
                                 maxit=args.maxit if args.mode == "pcg" else 10000)
    h = mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed, params=params)
    if args.form == "mixed":
        h.set_solver(mfto.FORMS[args.inner_form], args.inner_tol)
        h.set_cg_engine(args.cg_engine)
        h.set_ir_mode(IR_MODES[args.ir_mode])
        if args.kv_shape:
            h.set_kv_shape(*(int(x) for x in args.kv_shape.split(",")))
        elif not args.no_autotune:
            h.kv_autotune()
    f = torch.tensor(P.f, device=dev)
    u = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
    if args.mode == "profile":
        rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=dev)
        for _ in range(args.warmup + args.steps):
            h.simp_step(rho, u, f)
    else:
        rho = torch.tensor(W.rho_random(m, seed=1, lo=0.1, hi=1.0), device=dev)
        E = torch.empty_like(rho)
        h.simp_modulus(rho, E)
        st = h.pcg(E, f, u)
        print(json.dumps({"workload": args.workload, "cg_iterations": st.iterations,
                          "rel_residual": st.rel_residual}))
    torch.cuda.synchronize()
    h.close()


def kernel_case_run(args):
    """Short runs of one kernel family on a moderate case, for ncu captures of
    the kernels outside the benchmark's step (--case):
      tc      FP32-input K.v in each tensor-core form (3 launches each: TF32,
              split TF32, BF16, split BF16, FP16, split FP16) on --workload;
      multi   the 8-load-case mixed solve, 100 x 50 x 50 (inner CG capped);
      batch   the 64 uneven instances' batched mixed solve;
      nn      U-Net forward and gradient on the 136 x 72 x 40 node grid of a
              128 x 64 x 32 mesh (the learned part's training size), or forward
              passes on the node grid of --workload's mesh;
      simp    two SIMP iterations (filter, solve, compliance, OC) on --workload."""
    import numpy as np
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W
    dev = torch.device("cuda:0")
    case = args.case
    if case == "tc":
        P = W.WORKLOADS[args.workload]()
        m = P.mesh
        with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
            E = torch.tensor(W.rho_random(m, seed=1), dtype=torch.float32, device=dev) ** 3
            v = torch.tensor(W.vec_random(m.n_dof, seed=1), dtype=torch.float32, device=dev)
            y = torch.empty_like(v)
            for name in ("tf32", "tf32x3", "bf16", "bf16x3", "f16", "f16x3"):
                for _ in range(3):
                    h.kv(E, v, y, form=mfto.FORMS[name])
            torch.cuda.synchronize()
    elif case == "multi":
        P = W.WORKLOADS["cantilever_100x50x50_8rhs"]()
        m = P.mesh
        nr = P.f.shape[0]
        with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                         params=mfto.default_params(max_rhs=nr)) as h:
            h.set_solver(mfto.FORM_F32, 1e-1, 64, 1)
            h.set_ir_mode(IR_MODES["continue"])
            E = torch.full((m.n_elem,), 0.3 ** 3, dtype=torch.float64, device=dev)
            F = torch.tensor(P.f.reshape(-1), device=dev)
            U = torch.zeros(nr * m.n_dof, dtype=torch.float64, device=dev)
            h.ir_solve_multi(E, F, U, nr, inner_tol=1e-1)
            Y = torch.empty(nr * m.n_dof, dtype=torch.float32, device=dev)
            h.kv_multi(E.float(), U.float(), Y, nr, form=mfto.FORM_F32)
            torch.cuda.synchronize()
    elif case == "batch":
        probs = W.uneven_instances(count=64, seed=5)
        with mfto.Batch([(q.mesh.nelx, q.mesh.nely, q.mesh.nelz) for q in probs],
                        [q.fixed for q in probs]) as b:
            Eb = torch.full((b.n_elem,), 0.3 ** 3, dtype=torch.float64, device=dev)
            Fb = torch.tensor(np.concatenate([q.f for q in probs]), device=dev)
            Ub = torch.zeros(b.n_dof, dtype=torch.float64, device=dev)
            b.solve(Eb, Fb, Ub, inner_tol=1e-2, inner_maxit=64, max_outer=1)
            Y = torch.empty(b.n_dof, dtype=torch.float32, device=dev)
            b.kv(Eb.float(), Ub.float(), Y, form=mfto.FORM_F32)
            torch.cuda.synchronize()
    elif case == "nn":
        # the training mesh 128 x 64 x 32 by default (forward and gradient);
        # with --workload another mesh, forward passes only above 2M voxels
        mesh = (128, 64, 32)
        if args.workload != WORKLOAD:
            pm = W.WORKLOADS[args.workload]().mesh
            mesh = (pm.nelx, pm.nely, pm.nelz)
        dims = mfto.nn_grid(*mesh)
        V = int(np.prod(dims))
        train = V <= 2_000_000
        net = mfto.Net(base=14, levels=4, max_voxels=V, max_train_voxels=V if train else 0, seed=0)
        try:
            g = torch.Generator(device="cpu").manual_seed(0)
            x = torch.rand(4 * V, generator=g).to(dev)
            t = torch.rand(3 * V, generator=g).to(dev)
            mask = torch.ones(3 * V, device=dev)
            out = torch.empty(3 * V, device=dev)
            for _ in range(2):
                net.forward(x, out, dims)
                if train:
                    net.gradient(x, t, mask, dims)
            torch.cuda.synchronize()
        finally:
            net.close()
    elif case == "simp":
        P = W.WORKLOADS[args.workload]()
        m = P.mesh
        params = mfto.default_params(volfrac=P.volfrac, rmin=P.rmin, rtol=1e-8)
        with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed, params=params) as h:
            h.set_solver(mfto.FORM_F32, 1e-1)
            rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=dev)
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
            f = torch.tensor(P.f, device=dev)
            for _ in range(2):
                h.simp_step(rho, u, f)
            torch.cuda.synchronize()
    print(json.dumps({"case": case, "ok": True}))


def compare_run(args):
    """Forms side by side on the GPU, one JSON line each (plain FP64 is the
    reference; the oracle is not used here):
      torsion 55x55x165: SIMP iterations with plain FP64 and the mixed solve
        with every inner form and tolerance, from the same state;
      100x50x50 cantilever, 8 load cases: the multi-RHS mixed solve against
        8 single mixed solves and 8 plain FP64 solves;
      64 uneven cantilevers (16x8x8 .. 48x24x24): the batched mixed solve
        against 64 single mixed and 64 plain FP64 solves."""
    import numpy as np
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W
    dev = torch.device("cuda:0")
    out = []

    def sync_time(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    # ---- torsion: forms
    P = W.WORKLOADS["torsion_55x55x165"]()
    m = P.mesh
    h = mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                    params=mfto.default_params(volfrac=P.volfrac, rmin=P.rmin))
    rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=dev)
    u = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
    f = torch.tensor(P.f, device=dev)
    for _ in range(args.warmup):
        h.simp_step(rho, u, f)
    rho0, u0 = rho.clone(), u.clone()
    # (form, inner tolerance, refinement mode): the paper's tolerances with
    # restarted inner solves, and the continued-direction solve at 0.1
    forms = [("f64", None, "restart"), ("f32", 1e-1, "continue"), ("f32", 1e-2, "restart"),
             ("f32", 1e-4, "restart"), ("tf32x3", 1e-2, "restart"), ("f16x3", 1e-2, "restart"),
             ("bf16x3", 1e-2, "restart"), ("tf32", 1e-2, "restart"), ("f16", 1e-2, "restart"),
             ("bf16", 1e-2, "restart"), ("tf32x3", 1e-1, "continue"), ("f16x3", 1e-1, "continue")]
    h.kv_autotune()
    ref_c = None
    for name, tol, mode in forms:
        h.set_solver(mfto.FORMS[name], tol or 1e-2, 10000, 30)
        h.set_ir_mode(IR_MODES[mode])
        rho.copy_(rho0)
        u.copy_(u0)
        cs, ts, its, stat = [], [], [], []
        for _ in range(args.steps):
            dt, st = sync_time(lambda: h.simp_step(rho, u, f))
            cs.append(st.compliance)
            ts.append(dt)
            its.append(st.cg_iterations)
            stat.append(mfto.STATUS_NAMES[st.cg_status])
        if ref_c is None:
            ref_c = cs
        out.append({"case": "torsion_55x55x165", "form": name, "inner_tol": tol,
                    "refinement": mode if name != "f64" else None,
                    "simp_iter_ms": 1e3 * float(np.mean(ts)), "cg_iterations": its,
                    "solve_status": stat, "compliance": cs,
                    "compliance_rel_err_vs_f64": max(abs(a - b) / abs(b)
                                                     for a, b in zip(cs, ref_c))})
    h.close()

    # ---- 8 load cases
    P = W.WORKLOADS["cantilever_100x50x50_8rhs"]()
    m = P.mesh
    nr = P.f.shape[0]
    h = mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed, params=mfto.default_params(max_rhs=nr))
    h.kv_autotune()
    h.set_solver(mfto.FORM_F32, 1e-1, 10000, 50)
    h.set_ir_mode(IR_MODES["continue"])
    E = torch.full((m.n_elem,), 0.3 ** 3, dtype=torch.float64, device=dev)
    F = torch.tensor(P.f.reshape(-1), device=dev)
    U = torch.zeros(nr * m.n_dof, dtype=torch.float64, device=dev)
    h.ir_solve_multi(E, F, U, nr, inner_tol=1e-1)           # warm-up (graph capture)
    U.zero_()
    t_multi, sts = sync_time(lambda: h.ir_solve_multi(E, F, U, nr, inner_tol=1e-1))
    c_multi = [float(F[r * m.n_dof:(r + 1) * m.n_dof] @ U[r * m.n_dof:(r + 1) * m.n_dof])
               for r in range(nr)]
    t_single = t_f64 = 0.0
    c64 = []
    for r in range(nr):
        fr = F[r * m.n_dof:(r + 1) * m.n_dof].contiguous()
        ur = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
        h.ir_solve(E, fr, ur, inner_tol=1e-1)                # warm-up
        ur.zero_()
        dt, _ = sync_time(lambda: h.ir_solve(E, fr, ur, inner_tol=1e-1))
        t_single += dt
        ur.zero_()
        dt, _ = sync_time(lambda: h.pcg(E, fr, ur))
        t_f64 += dt
        c64.append(float(fr @ ur))
    # the multigrid solve of the 8 cases on one hierarchy
    h.gmg_solve_multi(E, F, U, nr)                       # warm-up (storage, graph captures)
    U.zero_()
    t_gmg, sts_g = sync_time(lambda: h.gmg_solve_multi(E, F, U, nr))
    c_gmg = [float(F[r * m.n_dof:(r + 1) * m.n_dof] @ U[r * m.n_dof:(r + 1) * m.n_dof])
             for r in range(nr)]
    out.append({"case": "cantilever_100x50x50_8rhs", "multi_rhs_mixed_s": t_multi,
                "gmg_multi_s": t_gmg, "gmg_statuses": [mfto.STATUS_NAMES[s.status] for s in sts_g],
                "gmg_iterations": [s.iterations for s in sts_g],
                "gmg_compliance_rel_err_vs_f64": max(abs(a - b) / abs(b)
                                                     for a, b in zip(c_gmg, c64)),
                "single_mixed_x8_s": t_single, "plain_f64_x8_s": t_f64,
                "statuses": [mfto.STATUS_NAMES[s.status] for s in sts],
                "max_rel_residual": max(s.rel_residual for s in sts),
                "compliance_rel_err_vs_f64": max(abs(a - b) / abs(b) for a, b in zip(c_multi, c64))})
    h.close()

    # ---- 64 uneven instances
    probs = W.uneven_instances(count=64, seed=5)
    with mfto.Batch([(p.mesh.nelx, p.mesh.nely, p.mesh.nelz) for p in probs],
                    [p.fixed for p in probs]) as b:
        shape, ms = b.autotune(reps=5)
        Eb = torch.full((b.n_elem,), 0.3 ** 3, dtype=torch.float64, device=dev)
        Fb = torch.tensor(np.concatenate([p.f for p in probs]), device=dev)
        Ub = torch.zeros(b.n_dof, dtype=torch.float64, device=dev)
        t_batch, c_batch, sts = {}, {}, {}
        offs = b.dof_off
        for mode, tol in (("restart", 1e-2), ("continue", 1e-1)):
            b.set_ir_mode(IR_MODES[mode])
            b.solve(Eb, Fb, Ub, inner_tol=tol)      # warm-up (graph capture)
            Ub.zero_()
            t_batch[mode], sts[mode] = sync_time(lambda: b.solve(Eb, Fb, Ub, inner_tol=tol))
            c_batch[mode] = [float(Fb[offs[i]:offs[i + 1]] @ Ub[offs[i]:offs[i + 1]])
                             for i in range(64)]
            Ub.zero_()
    t_single = {"restart": 0.0, "continue": 0.0}
    t_f64 = 0.0
    c64 = []
    for i, p in enumerate(probs):
        mm = p.mesh
        with mfto.Handle(mm.nelx, mm.nely, mm.nelz, p.fixed) as hs:
            Ei = torch.full((mm.n_elem,), 0.3 ** 3, dtype=torch.float64, device=dev)
            fi = torch.tensor(p.f, device=dev)
            ui = torch.zeros(mm.n_dof, dtype=torch.float64, device=dev)
            for mode, tol in (("restart", 1e-2), ("continue", 1e-1)):
                hs.set_ir_mode(IR_MODES[mode])
                hs.ir_solve(Ei, fi, ui, inner_tol=tol)   # warm-up
                ui.zero_()
                dt, _ = sync_time(lambda: hs.ir_solve(Ei, fi, ui, inner_tol=tol))
                t_single[mode] += dt
                ui.zero_()
            ui.zero_()
            hs.pcg(Ei, fi, ui)
            ui.zero_()
            dt, _ = sync_time(lambda: hs.pcg(Ei, fi, ui))
            t_f64 += dt
            c64.append(float(fi @ ui))
    for mode, tol in (("restart", 1e-2), ("continue", 1e-1)):
        out.append({"case": "64_uneven_cantilevers", "refinement": mode, "inner_tol": tol,
                    "autotuned_shape": shape, "shape_ms": [float(x) for x in ms],
                    "batched_mixed_s": t_batch[mode], "single_mixed_x64_s": t_single[mode],
                    "plain_f64_x64_s": t_f64,
                    "inner_iterations": sum(s.inner_iterations for s in sts[mode]),
                    "all_ok": all(s.status == mfto.OK for s in sts[mode]),
                    "compliance_rel_err_vs_f64": max(abs(a - b) / abs(b)
                                                     for a, b in zip(c_batch[mode], c64))})
    for o in out:
        print(json.dumps(o))


def learned_run(args):
    """The learned form at the 256 x 128 x 150 cantilever (4,915,200 elements,
    V_f 0.12): `warmup` SIMP iterations from the uniform start with the mixed
    solve, then, from that same state, `steps` SIMP iterations with each
    solver: plain FP64 Jacobi-PCG, the mixed solve, and the learned solve
    with the committed trained network and with an untrained one (initial
    guess only, every = 0).  One JSON line per solver: SIMP iteration time,
    inner iterations, network time, and the largest relative compliance
    difference to plain FP64."""
    import numpy as np
    import torch
    from paper_2604_18020_gb300 import learned as L, mfto, workloads as W
    dev = torch.device("cuda:0")
    nx, ny, nz, vf = 256, 128, 150, 0.12
    P = W.cantilever(nx, ny, nz)
    m = P.mesh
    V = int(np.prod(mfto.nn_grid(nx, ny, nz)))
    nets = {"learned_trained": L.load(L.WEIGHTS, V),
            "learned_untrained": mfto.Net(base=14, levels=4, max_voxels=V, seed=0)}
    h = mfto.Handle(nx, ny, nz, P.fixed,
                    params=mfto.default_params(volfrac=vf, rtol=1e-8, maxit=100000))
    h.set_solver(mfto.FORM_F32, args.inner_tol, 100000, 50)
    rho = torch.full((m.n_elem,), vf, dtype=torch.float64, device=dev)
    u = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
    f = torch.tensor(P.f, device=dev)
    for _ in range(args.warmup):
        h.simp_step(rho, u, f)
    rho0, u0 = rho.clone(), u.clone()
    h.kv_autotune()
    ref_c = None
    # the mixed solve as benchmarked (continued direction, inner tolerance
    # 0.1) and as the learned solve was designed against (restart, 1e-2)
    solvers = [("f64", None, "restart"), ("mixed", 1e-1, "continue"),
               ("mixed_restart", 1e-2, "restart"), ("learned_trained", 1e-2, "restart"),
               ("learned_untrained", 1e-2, "restart")]
    for name, tol, mode in solvers:
        h.set_learned(nets.get(name), every=0)
        h.set_solver(mfto.FORM_F64 if name == "f64" else mfto.FORM_F32, tol or 1e-2, 100000, 50)
        h.set_ir_mode(IR_MODES[mode])
        rho.copy_(rho0)
        u.copy_(u0)
        cs, ts, its = [], [], []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            st = h.simp_step(rho, u, f)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t)
            cs.append(st.compliance)
            its.append(st.cg_iterations)
        ref_c = ref_c or cs
        print(json.dumps({"case": "cantilever_256x128x150_vf0.12", "solver": name,
                          "inner_tol": tol, "refinement": mode if name != "f64" else None,
                          "warmup_simp_iters": args.warmup, "simp_iter_ms": 1e3 * float(np.mean(ts)),
                          "iterations": its, "compliance": cs,
                          "compliance_rel_err_vs_f64": max(abs(a - b) / abs(b)
                                                           for a, b in zip(cs, ref_c))}),
              flush=True)
    h.set_learned(None)
    h.close()


def unet_run(args):
    """U-Net timing, tensor-core convolutions against the FMA-pipe ones: the
    forward pass on the node grid of the learned workload's 256 x 128 x 150
    mesh (264 x 136 x 152 voxels) and forward + gradient on the training
    grid of a 128 x 64 x 32 mesh (136 x 72 x 40), base width 14, 4 levels;
    device time from CUDA events, median of 5 calls after 2 warm-ups.  One
    JSON line per grid and setting."""
    import numpy as np
    import torch
    from paper_2604_18020_gb300 import mfto
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()

    def timed(fn, reps=5, warm=2):
        for _ in range(warm):
            fn()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    def forward_flops(V, base=14, levels=4, cin=4, cout=3):
        # 2 flop per multiply-add: 27 taps per 3x3x3 layer, one per 1x1x1
        f, prev = 0, cin
        for l in range(levels - 1):                      # encoders
            c = base << l
            f += 2 * 27 * (prev * c + c * c) * (V >> (3 * l))
            prev = c
        cb, Vb = base << (levels - 1), V >> (3 * (levels - 1))
        f += 2 * 27 * (prev * cb + cb * cb) * Vb          # bottleneck
        for l in range(levels - 2, -1, -1):               # decoders
            c = base << l
            f += 2 * 27 * (((base << (l + 1)) + c) * c + c * c) * (V >> (3 * l))
        return f + 2 * base * cout * V                    # head

    for mesh, train in (((256, 128, 150), False), ((128, 64, 32), True)):
        dims = mfto.nn_grid(*mesh)
        V = int(np.prod(dims))
        net = mfto.Net(base=14, levels=4, max_voxels=V, max_train_voxels=V if train else 0, seed=0)
        try:
            g = torch.Generator(device="cpu").manual_seed(0)
            x = torch.rand(4 * V, generator=g).to(dev)
            t = torch.rand(3 * V, generator=g).to(dev)
            mask = torch.ones(3 * V, device=dev)
            out = torch.empty(3 * V, device=dev)
            for tc in (True, False):
                net.set_tensor_cores(tc)
                fwd = timed(lambda: net.forward(x, out, dims))
                rec = {"case": "unet_b14_l4", "grid": list(dims), "voxels": V,
                       "tensor_cores": tc, "forward_ms": fwd,
                       "forward_gflop": forward_flops(V) / 1e9}
                rec["forward_tflops"] = rec["forward_gflop"] / fwd
                if train:
                    # gradient: forward + backward, synchronised by the call
                    rec["gradient_ms"] = timed(lambda: net.gradient(x, t, mask, dims))
                rec["gave_up"] = net.tc_gave_up()
                print(json.dumps(rec), flush=True)
        finally:
            net.close()


def kappa_run(args):
    """kappa(K) on the free DOFs by power and inverse iteration (the paper's
    caps and tolerances, start vectors from seeds 42 and 123) for the paper's
    cantilever sizes at uniform density 0.5, p = 3 and 5; one JSON line each,
    with the paper's printed estimate for the size."""
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W
    dev = torch.device("cuda:0")
    paper = {64000: 6.1e5, 216000: 1.3e6, 512000: 2.3e6}
    for dims in ((80, 40, 20), (120, 60, 30), (160, 80, 40)):
        P = W.cantilever_point(*dims)
        m = P.mesh
        with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
            for penal in (3.0, 5.0):
                rho = torch.full((m.n_elem,), 0.5, dtype=torch.float64, device=dev)
                E = torch.empty_like(rho)
                h.set_params(mfto.default_params(penal=penal))
                h.simp_modulus(rho, E)
                vp = torch.tensor(W.vec_random(m.n_dof, seed=42), device=dev)
                vi = torch.tensor(W.vec_random(m.n_dof, seed=123), device=dev)
                torch.cuda.synchronize()
                t = time.perf_counter()
                st = h.kappa(E, vp, vi)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t
                print(json.dumps({
                    "case": f"cantilever_{dims[0]}x{dims[1]}x{dims[2]}", "elements": m.n_elem,
                    "penal": penal, "lambda_max": st.lambda_max, "lambda_min": st.lambda_min,
                    "kappa": st.kappa, "paper_kappa": paper[m.n_elem],
                    "power_steps": st.power_steps, "inverse_steps": st.inverse_steps,
                    "inner_iterations": st.inner_iterations, "inner_capped": st.inner_capped,
                    "seconds": dt}), flush=True)


def protocol_run(args):
    """The SIMP-120 continuation protocol (projection, four phases, restarts,
    selected iterate) on the paper's point-load cantilever of --workload's
    size, with the solvers of --protocol-solvers (mixed: FP32 Jacobi-PCG in
    FP64 refinement; f64: plain FP64 Jacobi-PCG; gmg: the multigrid solve):
    wall time, selected compliance and iteration counts, one JSON line each."""
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W
    dev = torch.device("cuda:0")
    base = W.WORKLOADS[args.workload]()
    m0 = base.mesh
    P = W.cantilever_point(m0.nelx, m0.nely, m0.nelz)
    m = P.mesh
    for solver in args.protocol_solvers.split(","):
        params = mfto.default_params(volfrac=P.volfrac, rmin=P.rmin, rtol=1e-8)
        with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed, params=params) as h:
            if solver in ("mixed", "gmg"):
                h.set_solver(mfto.FORM_F32, args.inner_tol)
                h.set_ir_mode(IR_MODES[args.ir_mode])
                tuned = h.kv_autotune()
            if solver == "gmg":                        # V-cycle CG (default parameters,
                h.set_gmg_solver(                      # Chebyshev sweeps if asked)
                    True, mfto.default_gmg_params(cheb_degree=args.gmg_cheb))
            rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=dev)
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
            f = torch.tensor(P.f, device=dev)
            sel = torch.zeros_like(rho)
            pp = mfto.default_protocol_params(n_iter=args.protocol_iters, rmin0=P.rmin)
            torch.cuda.synchronize()
            t = time.perf_counter()
            st, comp, gray, rest = h.simp_protocol(rho, u, f, sel, pp)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            print(json.dumps({
                "case": f"cantilever_point_{m.nelx}x{m.nely}x{m.nelz}", "elements": m.n_elem,
                "solver": solver + (f"_cheb{args.gmg_cheb}" if solver == "gmg" and
                                    args.gmg_cheb >= 0 else ""),
                "iterations": st.iterations, "seconds": dt,
                "ms_per_iteration": 1e3 * dt / st.iterations,
                "solver_iterations": st.cg_iterations, "restarts": st.restarts,
                "selected_iteration": st.selected_iteration,
                "selected_compliance": st.selected_compliance,
                "final_compliance": float(comp[-1]), "final_grayness": float(gray[-1])}),
                flush=True)


def hard_run(args):
    """The paper's hard problems (MBB, bridge, 150 x 50 x 25 = 187,500
    elements): cold-start FEA solves at the uniform initial density (p = 3;
    mean of 5 after one warm-up) and the 60-iteration cold-start SIMP runs of
    the protocol, each with plain FP64 Jacobi-PCG, the mixed solve and the
    multigrid solve; one JSON line per problem."""
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W
    dev = torch.device("cuda:0")
    for name in ("mbb_150x50x25", "bridge_150x50x25"):
        P = W.WORKLOADS[name]()
        m = P.mesh
        f = torch.tensor(P.f, device=dev)
        res = {}
        for solver in ("f64", "mixed", "gmg"):
            params = mfto.default_params(volfrac=P.volfrac, rmin=P.rmin, rtol=1e-8, maxit=20000)
            with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed, params=params) as h:
                if solver in ("mixed", "gmg"):
                    h.set_solver(mfto.FORM_F32, args.inner_tol, 20000, 80)
                    h.set_ir_mode(IR_MODES[args.ir_mode])
                    h.kv_autotune()
                if solver == "gmg":
                    h.set_gmg_solver(True)
                rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=dev)
                E = torch.empty_like(rho)
                rho_phys = torch.empty_like(rho)
                h.filter(rho, rho_phys)
                h.simp_modulus(rho_phys, E)
                u = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
                times, its, rel = [], [], []
                for rep in range(6):
                    u.zero_()
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    if solver == "f64":
                        st = h.pcg(E, f, u)
                        it = st.iterations
                    elif solver == "gmg":
                        st = h.gmg_solve(E, f, u)
                        it = st.iterations
                    else:
                        st = h.ir_solve(E, f, u, inner_tol=args.inner_tol)
                        it = st.inner_iterations
                    torch.cuda.synchronize()
                    if rep:
                        times.append(time.perf_counter() - t)
                        its.append(it)
                        rel.append(st.rel_residual)
                c_fea = float((f * u).sum())
                sel = torch.zeros_like(rho)
                rho.fill_(P.volfrac)
                u.zero_()
                pp = mfto.default_protocol_params(n_iter=60, rmin0=P.rmin, cold_start=1)
                torch.cuda.synchronize()
                t = time.perf_counter()
                pst, comp, gray, rest = h.simp_protocol(rho, u, f, sel, pp)
                torch.cuda.synchronize()
                t60 = time.perf_counter() - t
                res[solver] = {"fea_ms": 1e3 * sum(times) / len(times), "fea_iterations": its[-1],
                               "fea_rel_residual": rel[-1], "fea_compliance": c_fea,
                               "simp60_s": t60, "simp60_solver_iterations": pst.cg_iterations,
                               "simp60_selected_iteration": pst.selected_iteration,
                               "simp60_selected_compliance": pst.selected_compliance,
                               "simp60_restarts": pst.restarts}
        a, b = res["f64"], res["mixed"]
        g = res["gmg"]
        print(json.dumps({
            "case": name, "elements": m.n_elem, "f64": a, "mixed": b, "gmg": g,
            "gmg_fea_speedup_vs_f64": a["fea_ms"] / g["fea_ms"],
            "gmg_simp60_speedup_vs_f64": a["simp60_s"] / g["simp60_s"],
            "fea_speedup": a["fea_ms"] / b["fea_ms"], "simp60_speedup": a["simp60_s"] / b["simp60_s"],
            "fea_compliance_rel_diff": abs(b["fea_compliance"] - a["fea_compliance"]) / abs(a["fea_compliance"]),
            "simp60_selected_compliance_rel_diff":
                abs(b["simp60_selected_compliance"] - a["simp60_selected_compliance"])
                / abs(a["simp60_selected_compliance"]) if a["simp60_selected_iteration"] else None}),
            flush=True)


def ubench_run(args):
    """The synthetic hot-path microbenchmark of Sec. 5 (Tab. profiling) at
    its four sizes (cantilever shapes 80x40x20 .. 200x100x50, 64k .. 1M
    elements) on random element connectivity (seed 42): the staged FP64
    pipeline (gather, element contraction, scatter) and the fused FP64 and
    FP32 kernels, device times from CUDA events, median of the timed calls;
    beside them the structured-mesh K.v of the library (FP64 and the FP32
    column kernel, no atomics) on the same shapes.  One JSON line per size."""
    import numpy as np
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W
    dev = torch.device("cuda:0")
    reps = max(args.steps, 20)
    for shape in ((80, 40, 20), (120, 60, 30), (160, 80, 40), (200, 100, 50)):
        m = W.Mesh(*shape)
        edof = torch.tensor(W.edof_random(m, 42), device=dev)
        E64 = torch.tensor(W.rho_random(m, seed=1), device=dev)
        v64 = torch.tensor(W.vec_random(m.n_dof, seed=2), device=dev)
        E32, v32 = E64.float(), v64.float()
        y64 = torch.empty_like(v64)
        y32 = torch.empty_like(v32)
        row = {"case": "ubench_random_index", "mesh": "x".join(map(str, shape)),
               "elements": m.n_elem, "dofs": m.n_dof, "timed_calls": reps}
        with mfto.Ebe(m.n_elem, m.n_dof) as e:
            for variant, key in ((0, "staged_f64"), (1, "fused_f64"), (2, "fused_f32")):
                Ev, vv, yv = (E32, v32, y32) if variant == 2 else (E64, v64, y64)
                for _ in range(args.warmup):
                    e.kv(variant, edof, Ev, vv, yv, timed=True)
                ts = np.array([e.kv(variant, edof, Ev, vv, yv, timed=True) for _ in range(reps)])
                med = np.median(ts, axis=0) * 1e3
                if variant == 0:
                    row["t_gather_us"], row["t_contract_us"], row["t_scatter_us"] = map(float, med)
                    row["t_full64_us"] = float(np.median(ts.sum(axis=1)) * 1e3)
                else:
                    row[f"t_{key}_us"] = float(med[0])
        # the library's structured operator on the same shape (clamped x = 0 face)
        P = W.cantilever(*shape)
        with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
            h.kv_autotune()
            for form, key, Ev, vv, yv in ((mfto.FORM_F64, "structured_f64", E64, v64, y64),
                                          (mfto.FORM_F32, "structured_f32", E32, v32, y32)):
                for _ in range(args.warmup):
                    h.kv(Ev, vv, yv, form)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ts = []
                for _ in range(reps):
                    torch.cuda.synchronize()
                    ev0.record()
                    h.kv(Ev, vv, yv, form)
                    ev1.record()
                    torch.cuda.synchronize()
                    ts.append(ev0.elapsed_time(ev1))
                row[f"t_{key}_us"] = float(np.median(ts) * 1e3)
        row["fused_f32_speedup_vs_staged_f64"] = row["t_full64_us"] / row["t_fused_f32_us"]
        row["structured_f32_speedup_vs_staged_f64"] = row["t_full64_us"] / row["t_structured_f32_us"]
        print(json.dumps(row), flush=True)


def gmg_run(args):
    """Geometric multigrid against the Jacobi solvers on SIMP states (one
    JSON line per case): the 120x60x30 cantilever after 20 and the torsion
    problem after 10 SIMP iterations (mixed Jacobi solver, continued
    refinement), and the 256x128x150 cantilever at its uniform initial
    density; cold-start solves to rtol 1e-8 (mean of the timed calls after
    one warm-up), the hierarchy, the V-cycle time (CUDA events), and the
    time per SIMP iteration with each solver from the same state."""
    import numpy as np
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W
    dev = torch.device("cuda:0")

    def sync_time(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    reps = max(1, min(args.steps, 5))
    cases = (("cantilever_120x60x30", 20), ("torsion_55x55x165", 10),
             ("cantilever_256x128x150", 0))
    if args.gmg_case:
        cases = [(n, k if args.gmg_simp_iters is None else args.gmg_simp_iters)
                 for n, k in cases if n == args.gmg_case]
    for name, n_simp in cases:
        P = W.WORKLOADS[name]()
        m = P.mesh
        h = mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                        params=mfto.default_params(volfrac=P.volfrac, rmin=P.rmin))
        if not args.no_autotune:
            h.kv_autotune()
        h.set_solver(mfto.FORM_F32, 1e-1, 10000, 50)
        h.set_ir_mode(IR_MODES["continue"])
        rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=dev)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
        f = torch.tensor(P.f, device=dev)
        for _ in range(n_simp):
            h.simp_step(rho, u, f)
        rho_phys, E = torch.empty_like(rho), torch.empty_like(rho)
        h.filter(rho, rho_phys)
        h.simp_modulus(rho_phys, E)
        row = {"case": name, "elements": m.n_elem, "dofs": m.n_dof,
               "state": f"after {n_simp} SIMP iterations" if n_simp else "uniform initial density"}
        uu = torch.zeros_like(u)
        solvers = [("jacobi_f64", lambda: h.pcg(E, f, uu)),
                   ("jacobi_mixed_continue_0.1", lambda: h.ir_solve(E, f, uu, inner_tol=0.1))]
        gmg_cfg = [("gmg_f64", dict(mixed=0)), ("gmg_mixed", dict(mixed=1)),
                   ("gmg_mixed_l1", dict(mixed=1, cheb_degree=0)),
                   ("gmg_mixed_nu2", dict(mixed=1, nu_pre=2, nu_post=2, cheb_degree=0)),
                   ("gmg_mixed_restart", dict(mixed=1, continue_dir=0, cheb_degree=0)),
                   ("gmg_mixed_cheb2", dict(mixed=1, cheb_degree=2)),
                   ("gmg_mixed_cheb3", dict(mixed=1, cheb_degree=3))]
        # the fine sweeps on tensor-core K.v forms (a BF16 smoother inside a V-cycle)
        gmg_cfg += [(f"gmg_mixed_smoother_{fm}", dict(mixed=1, smoother_form=mfto.FORMS[fm]))
                    for fm in ("tf32", "bf16", "f16", "bf16x3")]
        if name == "cantilever_256x128x150":
            solvers = solvers[1:]                      # FP64 Jacobi: minutes at this size
        if args.gmg_only:                              # the default multigrid solve alone
            solvers, gmg_cfg = [], gmg_cfg[1:2]
        c_ref = None
        for key, fn in solvers + [(k, None) for k, _ in gmg_cfg]:
            if fn is None:
                prm = mfto.default_gmg_params(**dict(gmg_cfg)[key])
                h.set_gmg_solver(False, prm)
                fn = lambda: h.gmg_solve(E, f, uu)
            uu.zero_()
            fn()
            ts, st = [], None
            for _ in range(reps):
                uu.zero_()
                dt, st = sync_time(fn)
                ts.append(dt)
            its = st.inner_iterations if hasattr(st, "inner_iterations") else st.iterations
            c = float((f * uu).sum())
            c_ref = c if c_ref is None else c_ref
            row[key] = {"ms": 1e3 * float(np.mean(ts)), "iterations": its,
                        "status": mfto.STATUS_NAMES[st.status], "rel_residual": st.rel_residual,
                        "compliance_rel_diff": abs(c - c_ref) / abs(c_ref)}
        prm = mfto.default_gmg_params()
        h.set_gmg_solver(False, prm)
        dt, _ = sync_time(lambda: h.gmg_setup(E, prm))
        row["gmg_setup_ms"] = 1e3 * dt
        row["gmg_levels"] = h.gmg_levels()
        r32 = torch.tensor(W.vec_random(m.n_dof, seed=3), dtype=torch.float32, device=dev)
        z32 = torch.empty_like(r32)
        h.gmg_vcycle(r32, z32)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(20):
            h.gmg_vcycle(r32, z32)
        ev1.record()
        torch.cuda.synchronize()
        row["vcycle_ms"] = ev0.elapsed_time(ev1) / 20
        if args.gmg_only:
            h.close()
            print(json.dumps(row), flush=True)
            continue
        # SIMP iterations from the same state with each solver
        rho0, u0 = rho.clone(), u.clone()
        for key, use_gmg in (("simp_iter_ms_jacobi_mixed", False), ("simp_iter_ms_gmg_mixed", True)):
            h.set_gmg_solver(use_gmg, prm)
            rho.copy_(rho0)
            u.copy_(u0)
            ts, cs = [], []
            for _ in range(reps):
                dt, st = sync_time(lambda: h.simp_step(rho, u, f))
                ts.append(dt)
                cs.append(st.compliance)
            row[key] = 1e3 * float(np.mean(ts))
            row[key.replace("simp_iter_ms", "simp_compliances")] = cs
        h.set_gmg_solver(False)
        h.close()
        print(json.dumps(row), flush=True)


def scaling_run(args):
    """Cold-start FEA solves of the paper's point-load cantilever at uniform
    density 0.5 (p = 3) on its size ladder (216k, 512k, 1M, 2.0M, 4.9M, 8M
    elements: 120x60x30 .. 400x200x100) and one size beyond it (600x300x150,
    27M elements), to rtol 1e-8: plain FP64 Jacobi-PCG up to 1M, the mixed
    Jacobi solve up to 8M, the multigrid solve everywhere; mean of the timed
    calls after one warm-up, with the handle's device memory.  One JSON line
    per size."""
    import torch
    from paper_2604_18020_gb300 import mfto, workloads as W
    dev = torch.device("cuda:0")
    reps = max(1, min(args.steps, 3))
    sizes = [(120, 60, 30), (160, 80, 40), (200, 100, 50), (252, 126, 63), (340, 170, 85),
             (400, 200, 100), (600, 300, 150)]
    for shape in sizes:
        P = W.cantilever_point(*shape)
        m = P.mesh
        params = mfto.default_params(volfrac=P.volfrac, rmin=P.rmin, rtol=1e-8, maxit=50000)
        row = {"case": "cantilever_point_" + "x".join(map(str, shape)), "elements": m.n_elem,
               "dofs": m.n_dof}
        with mfto.Handle(*shape, P.fixed, params=params) as h:
            h.kv_autotune()
            h.set_solver(mfto.FORM_F32, 1e-1, 50000, 80)
            h.set_ir_mode(IR_MODES["continue"])
            E = torch.full((m.n_elem,), 0.5 ** 3, dtype=torch.float64, device=dev)
            f = torch.tensor(P.f, device=dev)
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
            solvers = [("gmg_mixed", lambda: h.gmg_solve(E, f, u))]
            if m.n_elem <= 8_000_000:
                solvers.insert(0, ("jacobi_mixed", lambda: h.ir_solve(E, f, u, inner_tol=0.1)))
            if m.n_elem <= 1_000_000:
                solvers.insert(0, ("jacobi_f64", lambda: h.pcg(E, f, u)))
            c_ref = None
            for key, fn in solvers:
                u.zero_()
                fn()
                ts = []
                for _ in range(reps):
                    u.zero_()
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    st = fn()
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t)
                its = st.inner_iterations if hasattr(st, "inner_iterations") else st.iterations
                c = float((f * u).sum())
                c_ref = c if c_ref is None else c_ref
                row[key] = {"s": sum(ts) / len(ts), "iterations": its,
                            "status": mfto.STATUS_NAMES[st.status],
                            "rel_residual": st.rel_residual,
                            "compliance_rel_diff": abs(c - c_ref) / abs(c_ref)}
            free_b, total_b = torch.cuda.mem_get_info(dev)
            row["library_bytes"] = h.device_bytes()
            row["device_used_bytes"] = int(total_b - free_b)
            row["gmg_levels"] = len(h.gmg_levels())
        del E, f, u
        torch.cuda.empty_cache()
        print(json.dumps(row), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-maxit", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="bench",
                    choices=["bench", "profile", "pcg", "cgkv", "kernels", "compare", "learned",
                             "kappa", "protocol", "hard", "ubench", "gmg", "scaling", "unet"])
    ap.add_argument("--case", default="simp", choices=["tc", "multi", "batch", "nn", "simp"],
                    help="--mode kernels: the kernel family to run")
    ap.add_argument("--protocol-iters", type=int, default=120)
    ap.add_argument("--protocol-solvers", default="mixed,f64",
                    help="--mode protocol: comma-separated solvers among mixed, f64, gmg")
    ap.add_argument("--gmg-case", default=None,
                    choices=["cantilever_120x60x30", "torsion_55x55x165", "cantilever_256x128x150"],
                    help="--mode gmg: run this case only")
    ap.add_argument("--gmg-simp-iters", type=int, default=None,
                    help="--mode gmg: SIMP iterations before the solves (default per case)")
    ap.add_argument("--gmg-cheb", type=int, default=-1,
                    help="--mode protocol: Chebyshev degree of the multigrid sweeps (0: l1-Jacobi, "
                         "-1: the library's automatic choice)")
    ap.add_argument("--gmg-only", action="store_true",
                    help="--mode gmg: the default multigrid solve and V-cycle only")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--form", default="mixed", choices=["f64", "mixed"],
                    help="f64: plain FP64 Jacobi-PCG; mixed: FP64 iterative refinement "
                         "around an FP32 inner PCG")
    ap.add_argument("--inner-tol", type=float, default=1e-1)
    ap.add_argument("--ir-mode", default="continue", choices=sorted(IR_MODES),
                    help="inner CG at each outer step: restart (p = z) or continue the direction")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default z-chunk of the FP32 column K.v")
    ap.add_argument("--kv-shape", default=None,
                    help="NZC,KIND: pin the FP32 column K.v launch shape instead of autotuning")
    ap.add_argument("--cg-engine", type=int, default=2, choices=[0, 1, 2],
                    help="FP32 inner CG: 0 per-iteration graph, 1 persistent cooperative kernel, "
                         "2 per-iteration graph without grid tickets")
    ap.add_argument("--inner-form", default="f32",
                    choices=["f32", "tf32", "tf32x3", "bf16", "bf16x3", "f16", "f16x3"],
                    help="K.v form of the inner solve of --form mixed")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the FP32 CG K.v timing on the 256x128x150 cantilever")
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-extra", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--maxit", type=int, default=40, help=argparse.SUPPRESS)
    args = ap.parse_args()

    if args.cpu_sample:
        res = cpu_sample(args.cpu_sample, args.steps, args.maxit)
        if args.cpu_extra:
            res["all_cores"] = cpu_allcores_kv(args.cpu_sample)
            res["simp_cfg0"] = cpu_simp_cfg0()
        print(json.dumps(res))
        return

    if args.mode == "compare":
        compare_run(args)
        return
    if args.mode == "kernels":
        kernel_case_run(args)
        return
    if args.mode == "learned":
        learned_run(args)
        return
    if args.mode == "unet":
        unet_run(args)
        return
    if args.mode == "kappa":
        kappa_run(args)
        return
    if args.mode == "protocol":
        protocol_run(args)
        return
    if args.mode == "hard":
        hard_run(args)
        return
    if args.mode == "ubench":
        ubench_run(args)
        return
    if args.mode == "gmg":
        gmg_run(args)
        return
    if args.mode == "scaling":
        scaling_run(args)
        return
    if args.mode == "cgkv":
        # the FP32 CG K.v alone on --workload (inner CG capped at --maxit)
        import torch
        dev = torch.device("cuda:0")
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        shape = tuple(int(x) for x in args.kv_shape.split(",")) if args.kv_shape else None
        print(json.dumps(large_kv_leg(dev, 2070.0, n_sm, args.maxit, args.workload, shape,
                                      args.cg_engine)))
        return
    if args.mode != "bench":
        profile_run(args)
        return

    rank, local_rank, world = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        # the oracle as it stands, on the host cores: warm-up steps untimed
        res = run_cpu_sample(WORKLOAD, args.warmup + args.steps, args.cpu_maxit)
        times, kvs = res["times"][args.warmup:], res["kv"][args.warmup:]
        value = res["n_elem"] * sum(kvs) / sum(times) / 1e9
        base = cpu_baseline_entry({"times": times, "kv": kvs, "n_elem": res["n_elem"]},
                                  args.cpu_maxit)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": "Gelem/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "f64", "pcg_maxit": args.cpu_maxit},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "Gelem/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}))
        return

    out = gpu_bench(args, rank, local_rank, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            res = run_cpu_sample(WORKLOAD, 1, args.cpu_maxit, extra=True)
            out["cpu_baseline"] = cpu_baseline_entry(res, args.cpu_maxit)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
