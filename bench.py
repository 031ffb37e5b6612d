#!/usr/bin/env python3
"""Benchmark of the Laplacian-preconditioned Schur solve inside one full
one-way SIMPLE-IBM time step on GB300.

Workload (default): 256^3 MAC grid on the unit cube, eight spheres with radii
uniform in [0.05, 0.1] at seeded non-overlapping positions, 60000 Fibonacci
markers split by area, random rigid marker velocities in [-1, 1], a smooth
random body force (8 sine modes), Re 200, dt 1e-3, first step from rest,
FGMRES to a relative residual of 1e-8.

A step = marker binning (ibm_set_markers) + ibm_step (predictor, correction
right-hand sides, Schur solve, force recovery, update, diagnostics): every
row of the hot path, one Schur solve per step, so steps/s = Schur solves/s.
The headline `value` uses the mixed form (FP32 V-cycle, FP32 Arnoldi cycles
refined by the FP64 true residual); beside it the same step with the FP64
outer iteration and the FP32 V-cycle, the plain FP64 form (FP64 V-cycle and
Arnoldi), the solve alone, and (from the oracle leg) each form's error
against the oracle's step solved to 1e-13.

`--profile-step` runs one warm-up step and then one step bracketed by
cudaProfilerStart/Stop (for `ncu --profile-from-start off`), and exits.

Multi-GPU: replicas only (one independent workload per rank, no collective on
the data path); `value` sums the ranks' step rates over the slowest rank's
time.  `--impl reference` times whole steps of the CPU oracle on the same
workload (rank 0 only).
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

METRIC = "Schur solves/s at 256^3 to 1e-8 residual, FP32-precond vs FP64; HBM fraction"
UNIT = "solves/s"

# DRAM traffic / algorithmic bytes of each timed kernel class: ncu's
# dram__bytes_read.sum + dram__bytes_write.sum of the class's kernels, each
# captured alone (one launch, one pass) in one step of the 256^3 eight-sphere
# workload, over the algorithmic bytes of those launches.  The profile
# summary keeps the commands and the per-launch numbers.  A class whose kernel
# changes after the capture must be removed here (its traffic then reads
# null).  Below 1: part of a launch's output is still in the 129 MB L2 when
# it ends (written back later, often never: the next kernel reads it there).
NCU_TRAFFIC_RATIO = {
    # predictor FP32 Chebyshev step (mode 1): 631.7 + 181.4 MB for 808.5 MB
    "helm_sweep": 1.0058,
    # finest-level smoothing, one V-cycle: k_first_v4 67.2 + 27.1 MB and the
    # two k_sweep_v4 134.2 + 38.8 and 134.2 + 37.4 MB, for 134.2 + 2 x 201.3 MB
    "mg_smooth_fine": 0.8177,
    # FP32 Gram-Schmidt at basis lengths 6 and 7
    "multidot": 1.0042,
    "axpy_norm": 0.9744,
    # Schur Laplacian class per step: 14 k_lap_ds (69.4 + 24.2 MB for 134.2 MB)
    # and 2 k_laplacian_fx forming b - L x (268.5 + 108.4 MB for 402.7 MB)
    "laplacian_f64": 0.7691,
    # marker terms of one FP32-cycle Schur product: k_marker_grad_interp_f32
    # 8.8 MB and k_shell_gradt_f32 70.2 + 0.8 MB, for 78.0 MB
    "schur_markers": 1.0219,
}


def max_over_ranks(ms, dist, device):
    """The slowest rank's time per step (the job ends with it); ms itself
    without a process group."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, ms):
    """Whole-job solves/s: each of the world ranks (replicas, no collective on
    the data path) completes one solve per step of ms milliseconds."""
    return world * 1000.0 / ms


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# Kernel classes reported in the bench line: label -> the library's profile
# class.  The library counts each class's algorithmic bytes per launch (every
# array read or written once; Gram-Schmidt from the actual basis length of each
# launch and the element size of the Arnoldi form; the V-cycle and the solve
# as the sum over the kernels they launch).  SOLVE_CLASSES are the parts of
# the Schur solve (the metric's unit); the roofline record names the one of
# them that takes the most time.
ROOFLINE_CLASSES = {
    "k_helm_cheb_v4 (predictor FP32 Chebyshev step: read e, e_old, r; write e_new)":
        "helm_sweep",
    "k_multidot_sp4 (Gram-Schmidt multi-dot on FP32 vectors, float4: w and V_0..V_j)":
        "multidot",
    "k_axpy_norm_sp4 (Gram-Schmidt axpy+norm on FP32 vectors, float4: V_0..V_j, w in/out)":
        "axpy_norm",
    ("Schur Laplacian class: k_lap_ds<float> (FP32 z in, exact product rounded to FP32 "
     "out) per iteration and k_laplacian_fx (FP64, stencil sum exact in 64-bit integers) "
     "of the FP64 true residuals"):
        "laplacian_f64",
    ("Schur marker terms: k_marker_grad_interp (t = 2 R^T G z per marker) and the B^T t "
     "gather on the shell cells (k_shell_gradt_f32 in the FP32 Arnoldi cycles, FP64 "
     "k_shell_gradt in the true residuals)"): "schur_markers",
    "k_first_v4 + k_sweep_v4 (finest V-cycle smoothing)": "mg_smooth_fine",
    "whole V-cycle (every level, the one-block coarse chain and the coarsest solve)": "vcycle",
}
SOLVE_CLASSES = ("multidot", "axpy_norm", "laplacian_f64", "schur_markers", "mg_smooth_fine")


def roofline(prof, steps, hbm, peak_kind):
    """Per-class achieved bandwidth (algorithmic bytes over the class's
    event-timed duration), the roofline record of the Schur-solve class that
    takes the most time, and the whole solve's record.  prof: class ->
    {"ms", "launches", "bytes"} summed over the timed steps."""
    classes = {}
    for name, cls in ROOFLINE_CLASSES.items():
        t_ms = prof[cls]["ms"]
        tot_bytes = prof[cls]["bytes"]
        n_l = max(1, prof[cls]["launches"])
        gbs = tot_bytes / (t_ms * 1e-3) / 1e9 if t_ms > 0 else 0.0
        classes[name] = {"ms_per_step": t_ms / steps, "launches_per_step": n_l / steps,
                         "achieved_gbs": gbs, "frac": gbs / hbm,
                         "bytes_per_launch": tot_bytes / n_l, "avg_launch_ms": t_ms / n_l}
    solve_names = [kk for kk, cls in ROOFLINE_CLASSES.items() if cls in SOLVE_CLASSES]
    best = max(solve_names, key=lambda kk: classes[kk]["ms_per_step"])
    cb = classes[best]
    cls = ROOFLINE_CLASSES[best]
    roof = {"bound": "hbm", "kernel": best, "achieved": cb["achieved_gbs"], "peak": hbm,
            "unit": "GB/s", "frac": cb["frac"], "peak_kind": peak_kind,
            "traffic": (NCU_TRAFFIC_RATIO[cls] * cb["bytes_per_launch"]
                        if cls in NCU_TRAFFIC_RATIO else None),
            "traffic_source": ("ncu DRAM bytes per algorithmic byte of the class's kernels, "
                               "each captured alone in one step at 256^3, times this "
                               "launch's algorithmic bytes"),
            "avg_launch_ms": cb["avg_launch_ms"],
            "bytes_per_launch": cb["bytes_per_launch"]}
    sv = prof["solve"]
    n_sv = max(1, sv["launches"])
    sv_gbs = sv["bytes"] / (sv["ms"] * 1e-3) / 1e9 if sv["ms"] > 0 else 0.0
    solve = {"what": ("the whole Schur solve (the metric's unit): algorithmic bytes of every "
                      "kernel it launches (V-cycles, Schur products, Gram-Schmidt, updates, "
                      "FP64 true residuals) over its event-timed duration"),
             "bytes_per_solve": sv["bytes"] / n_sv, "ms_per_solve": sv["ms"] / n_sv,
             "achieved": sv_gbs, "peak": hbm, "unit": "GB/s", "frac": sv_gbs / hbm,
             "peak_kind": peak_kind}
    return roof, classes, solve


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # nvidia-smi's start-up (driver and NVML initialisation) can stall the
        # CUDA calls of this process for tens of milliseconds: wait for its
        # first sample so that the start-up is over before the timed region
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 10.0 and self.proc.poll() is None:
            if Path(self.path).stat().st_size > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in Path(self.path).read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        rows = rows[1:]     # the first sample precedes the timed region
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def oracle_step(W, rtol=1e-8):
    """One whole oracle step of the workload on the host cores (marker
    operators, predictor, right-hand sides, FGMRES with the exact L^+ to rtol,
    force recovery, update, diagnostics), timed on the wall clock.  Returns
    (seconds, the oracle's step dict, worker threads)."""
    from oracle import mac, step
    workers = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    g = mac.Grid(W.n)
    out = step.step(g, W.Re, W.dt, W.X, W.U_gamma, W.f_body, rtol=rtol, workers=workers)
    return time.perf_counter() - t0, out, workers


def oracle_errors(ref, got):
    """Errors of a GPU step's (u, p, F) against the oracle's: relative 2-norm
    of the difference, the largest element difference relative to the
    largest element of the oracle's field, and the same on the shell cells
    (cells coupled to the markers through B = R^T G) and shell faces (faces
    in the support of R), where the marker terms act."""
    import numpy as np
    sysm = ref["sys"]
    g = sysm.g
    shell_f = np.unique(sysm.R.tocoo().row)
    ind = np.zeros(g.n_faces)
    ind[shell_f] = 1.0
    cells = np.zeros((g.nz, g.ny, g.nx), dtype=bool)
    for d, comp in enumerate(g.split_faces(ind)):
        ax = 2 - d
        nd = comp.shape[ax] - 1
        cells |= np.take(comp, np.arange(nd), axis=ax) > 0
        cells |= np.take(comp, np.arange(1, nd + 1), axis=ax) > 0
    shell_c = np.flatnonzero(cells.ravel())
    res = {}
    for key, sel in (("u", shell_f), ("p", shell_c), ("F", None)):
        a = np.asarray(got[key], dtype=np.float64)
        b = np.asarray(ref[key], dtype=np.float64)
        d = np.abs(a - b)
        e = {"rel_l2": float(np.linalg.norm(a - b) / np.linalg.norm(b)),
             "max_abs_rel": float(d.max() / np.abs(b).max())}
        if sel is not None and sel.size:
            e["shell_max_abs_rel"] = float(d[sel].max() / np.abs(b).max())
        res[key] = e
    return res


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def workload_config(W):
    nb = len(W.radii)
    bodies = (f"1 sphere r {W.radii[0]:g}" if nb == 1 else
              f"{nb} spheres r {W.info.get('radius_law', 'in [%.3f,%.3f]' % (W.radii.min(), W.radii.max()))}")
    cell_mb = 8.0 * W.n ** 3 / 1e6
    if cell_mb > 129.0:
        l2 = (f"no flush: one step streams tens of GB (FP64 fields {cell_mb:.0f}-"
              f"{3 * cell_mb:.0f} MB, Krylov basis GBs) through the 129 MB L2, so no step "
              f"starts with the previous step's data resident")
    else:
        l2 = f"small case: an FP64 cell field ({cell_mb:.1f} MB) fits in the 129 MB L2"
    return {"workload": f"{W.name}: {W.n}^3 MAC grid, {bodies}, {W.n_markers} markers "
                        f"(spacing ratio {W.info['spacing_ratio']:.2f}), Re {W.Re:g}, "
                        f"dt {W.dt:g}, first step from rest, FGMRES rtol 1e-8",
            "grid": [W.n, W.n, W.n], "markers": W.n_markers, "bodies": nb,
            "Re": W.Re, "dt": W.dt, "rtol": 1e-8, "l2": l2,
            "parallelism": "replicas"}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from paper_2501_15314_gb300 import workloads as wl
    W = wl.config(args.config, secondary=True)
    for _ in range(args.warmup):
        oracle_step(W)
    secs, iters = [], []
    for _ in range(args.steps):
        t, out, cores = oracle_step(W)
        secs.append(t)
        iters.append(int(out["iters"]))
        del out
    value = len(secs) / sum(secs)
    sample = (f"whole oracle steps at the full workload, each timed on the wall clock: "
              f"marker operators, predictor, right-hand sides, FGMRES with the exact L^+ "
              f"(DCT) to rtol 1e-8 ({min(iters)}-{max(iters)} iterations, all run), force "
              f"recovery, update, diagnostics; scipy.fft workers = {cores}, sparse products "
              f"single-threaded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(W),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2501_15314_gb300 import _lib
    from paper_2501_15314_gb300 import workloads as wl
    from paper_2501_15314_gb300.api import IBMSolver

    W = wl.config(args.config, secondary=True)
    n = W.n
    s = IBMSolver(n, Re=W.Re, dt=W.dt)
    lib = s.lib
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    X = dev(W.X)
    U = dev(W.U_gamma.ravel())
    f = dev(W.f_body)
    nf, m, k = s.nf, s.m, 3 * W.n_markers
    zf, zc, zk = (torch.zeros(nf, dtype=torch.float64, device="cuda"),
                  torch.zeros(m, dtype=torch.float64, device="cuda"),
                  torch.zeros(k, dtype=torch.float64, device="cuda"))
    out = dict(u=torch.empty_like(zf), p=torch.empty_like(zc), F=torch.empty_like(zk))
    stream = s.stream

    def step(prec, arnoldi=_lib.IBM_ARNOLDI_FP32):
        s.set_markers(X)
        _, st = s.step(zf, zf, zc, zk, U, f, out=out, precond_prec=prec, arnoldi=arnoldi,
                       rtol=1e-8)
        return st

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(fn, K):
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = [fn() for _ in range(K)]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / K, dist, "cuda")
        return ms, stats

    # ---- mixed form (headline) ----
    for _ in range(args.warmup):
        step(_lib.IBM_PREC_FP32)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = lib.ibm_kernel_launches()
    ms_mixed, st_mixed = timed(lambda: step(_lib.IBM_PREC_FP32), args.steps)
    launches = lib.ibm_kernel_launches() - l0
    clk = clocks.stop()
    # Kernel classes: a second timed pass of the same K steps with the
    # library's CUDA events around each class's launches.  The events sit
    # between launches in the stream, cost host time at every synchronisation
    # and break the programmatic-dependent-launch overlap of the kernels they
    # separate, so the headline pass above runs without them.
    s.profile_enable(True)
    ms_prof, _ = timed(lambda: step(_lib.IBM_PREC_FP32), args.steps)
    prof = s.profile_read()
    s.profile_enable(False)
    # each form's step result (every timed step repeats the same step), kept
    # on the host for the comparison with the oracle's solution
    to_host = lambda: {kk: v.cpu().numpy().copy() for kk, v in out.items()}  # noqa: E731
    results = {"headline_fp32_vcycle_fp32_arnoldi": to_host()}

    # ---- FP64 outer iteration with the FP32 V-cycle (FP64 Arnoldi) ----
    k64 = max(1, args.steps // 2)
    step(_lib.IBM_PREC_FP32, _lib.IBM_ARNOLDI_FP64)
    ms_ns, st_ns = timed(lambda: step(_lib.IBM_PREC_FP32, _lib.IBM_ARNOLDI_FP64), k64)
    results["fp32_vcycle_fp64_arnoldi"] = to_host()

    # ---- FP64 form (FP64 V-cycle, FP64 Arnoldi) ----
    step(_lib.IBM_PREC_FP64, _lib.IBM_ARNOLDI_FP64)
    ms_fp64, st_fp64 = timed(lambda: step(_lib.IBM_PREC_FP64, _lib.IBM_ARNOLDI_FP64), k64)
    results["fp64_form"] = to_host()

    # ---- the solve alone, on a right-hand side of the step's form ----
    a = 1.5 / W.dt
    s.set_markers(X)
    rhs_F = a * (s.interp(f) - U)
    b = a * s.gradient_t(f) + 2.0 * s.gradient_t(s.spread(rhs_F))
    solve_only = {}
    for name, prec, arn in (("fp32_vcycle_ds_arnoldi", _lib.IBM_PREC_FP32, _lib.IBM_ARNOLDI_DS),
                            ("fp32_vcycle_fp32_arnoldi", _lib.IBM_PREC_FP32,
                             _lib.IBM_ARNOLDI_FP32),
                            ("fp32_vcycle_fp64_arnoldi", _lib.IBM_PREC_FP32,
                             _lib.IBM_ARNOLDI_FP64),
                            ("fp64_vcycle_fp64_arnoldi", _lib.IBM_PREC_FP64,
                             _lib.IBM_ARNOLDI_FP64)):
        kw = dict(precond_prec=prec, arnoldi=arn, rtol=1e-8)
        s.solve_schur(b, **kw)
        msq, stq = timed(lambda: s.solve_schur(b, **kw)[1], k64)
        solve_only[name] = {"solves_per_s": job_rate(world, msq), "ms": msq,
                            "iters": stq[-1]["iters"], "relres": stq[-1]["relres_true"]}

    # ---- end to end through the public API with host buffers ----
    # Every step copies its inputs from pinned host memory and its results
    # back.  The copies run on two more streams, one per direction (the link
    # is full duplex), pipelined with the steps: step k+1's inputs go in and
    # step k-1's results come out while step k computes (two device buffer
    # sets, ordered by events).
    # The inputs travel in one pinned staging buffer and one device buffer per
    # set, the results likewise (every array a 256-byte-aligned view into
    # them): one copy per direction and step, so the host spends little time
    # issuing copies between steps (each step ends with a host
    # synchronisation, and the GPU waits while the host issues the next
    # launches).
    def packed(arrays, device, pinned):
        offs, total = {}, 0
        for kk, v in arrays.items():
            offs[kk] = total
            total += (v.numel() + 31) // 32 * 32          # 32 doubles = 256 bytes
        buf = torch.empty(total, dtype=torch.float64, device=device)
        if pinned:
            buf = buf.pin_memory()
        views = {kk: buf[offs[kk]:offs[kk] + v.numel()] for kk, v in arrays.items()}
        return buf, views

    srcs = dict(X=X.reshape(-1), U=U, f=f, u_n=zf, u_nm1=zf, p_n=zc, F_n=zk)
    hbuf_in, h_in = packed(srcs, "cpu", True)
    for kk, v in srcs.items():
        h_in[kk].copy_(v.cpu())
    dset_in = [packed(srcs, "cuda", False) for _ in range(2)]
    d_in = [dict(v, X=v["X"].view(3, -1)) for _, v in dset_in]
    dset_out = [packed(out, "cuda", False) for _ in range(2)]
    d_out = [v for _, v in dset_out]
    hset_out = [packed(out, "cpu", True) for _ in range(2)]
    h2d = sum(v.numel() * v.element_size() for v in h_in.values())
    d2h = sum(v.numel() * v.element_size() for v in hset_out[0][1].values())
    cstream = torch.cuda.Stream()           # host to device
    ostream = torch.cuda.Stream()           # device to host
    ev = lambda: torch.cuda.Event()  # noqa: E731
    ev_in, ev_done, ev_outc = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    for q in range(2):
        ev_done[q].record(stream)
        ev_outc[q].record(stream)

    def copy_in(b):
        with torch.cuda.stream(cstream):
            cstream.wait_event(ev_done[b])          # the step that last read buffer b
            dset_in[b][0].copy_(hbuf_in, non_blocking=True)
            ev_in[b].record(cstream)

    def copy_out(b):
        with torch.cuda.stream(ostream):
            ostream.wait_event(ev_done[b])
            hset_out[b][0].copy_(dset_out[b][0], non_blocking=True)
            ev_outc[b].record(ostream)

    def e2e_run(K):
        copy_in(0)
        stats = []
        for k in range(K):
            b = k & 1
            if k + 1 < K:
                copy_in(1 - b)                      # inputs of step k+1
            stream.wait_event(ev_in[b])
            stream.wait_event(ev_outc[b])           # results of step k-2 are out
            s.set_markers(d_in[b]["X"])
            _, st = s.step(d_in[b]["u_n"], d_in[b]["u_nm1"], d_in[b]["p_n"], d_in[b]["F_n"],
                           d_in[b]["U"], d_in[b]["f"], out=d_out[b],
                           precond_prec=_lib.IBM_PREC_FP32, rtol=1e-8)
            ev_done[b].record(stream)
            copy_out(b)
            stats.append(st)
        for q in range(2):
            stream.wait_event(ev_outc[q])           # every result is on the host
        return stats

    e2e_run(2)
    # the host link's rate on this machine (one input set in, one result set out)
    torch.cuda.synchronize()
    c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    with torch.cuda.stream(cstream):
        c0.record(cstream)
        dset_in[0][0].copy_(hbuf_in, non_blocking=True)
        c1.record(cstream)
        hset_out[0][0].copy_(dset_out[0][0], non_blocking=True)
        c2.record(cstream)
    torch.cuda.synchronize()
    h2d_gbs = h2d / (c0.elapsed_time(c1) * 1e6)
    d2h_gbs = d2h / (c1.elapsed_time(c2) * 1e6)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")

    # ---- adjoint of the step (transposed Schur solve) ----
    adjoint = adjoint_bench(s, W, X, U, f, out, zf, zc, zk, timed, k64)
    c_modes = cmode_bench(timed, max(1, k64 // 2))
    porous = porous_bench(timed, k64)
    fsi = ({"spread_force_criterion": fsi_bench(args.fsi_steps, args.fsi_xi, 1),
            "marker_force_criterion": fsi_bench(args.fsi_steps, args.fsi_xi, 0)}
           if args.fsi_steps > 0 else None)
    multistep = multistep_bench()

    # ---- roofline of the dominant kernel class ----
    hbm, peak_kind = measured_peaks()
    roof, classes, solve_roof = roofline(prof, args.steps, hbm, peak_kind)
    breakdown = {kk: {"ms_per_step": v["ms"] / args.steps, "launches": v["launches"]}
                 for kk, v in prof.items() if v["launches"]}

    value = job_rate(world, ms_mixed)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_mixed,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 V-cycle + f32 Arnoldi cycles (Schur product, marker terms included, "
                     "rounded to f32) refined by the f64 true residual; double-single "
                     "predictor; f64 iterate, residual and update",
            "data": "synthetic",
            "config": workload_config(W),
            "fp64_form": {"value": job_rate(world, ms_fp64), "unit": UNIT, "ms_per_step": ms_fp64,
                          "iters": st_fp64[-1]["iters"],
                          "relres_true": st_fp64[-1]["relres_true"],
                          "what": "FP64 V-cycle + FP64 Arnoldi, same step"},
            "fp32_vcycle_fp64_arnoldi": {
                "value": job_rate(world, ms_ns), "unit": UNIT, "ms_per_step": ms_ns,
                "iters": st_ns[-1]["iters"], "relres_true": st_ns[-1]["relres_true"],
                "what": ("same step; outer FGMRES, residuals and Schur products in FP64, "
                         "V-cycle preconditioner in FP32 with FP32 accumulation")},
            "solve_only": solve_only,
            "iters": st_mixed[-1]["iters"], "relres_true": st_mixed[-1]["relres_true"],
            "helm_iters": st_mixed[-1]["helm_iters"],
            "div_l2": st_mixed[-1]["div_l2"], "slip_l2": st_mixed[-1]["slip_l2"],
            "roofline": roof, "solve_roofline": solve_roof, "kernel_classes": classes,
            "profiled_pass": {
                "ms_per_step": ms_prof,
                "what": ("the kernel classes, the roofline records and the breakdown are "
                         "timed by CUDA events on the launching streams in a second pass of "
                         "the same K steps right after the headline pass; the events break "
                         "the programmatic-dependent-launch overlap and cost host time, so "
                         "this pass runs slower than the headline")},
            "breakdown": breakdown,
            "adjoint": adjoint, "c_modes": c_modes, "porous": porous, "two_way_fsi": fsi,
            "multistep": multistep,
            "gpu_launches": int(launches),
            "clocks": clk,
            "e2e": {"value": job_rate(world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                    "copies": "one pinned host buffer per direction (the step's seven input "
                              "arrays, its three results), one copy each way per step; H2D "
                              "and D2H each on a stream of its own, pipelined with the steps "
                              "(double-buffered)",
                    "h2d_gbs_alone": h2d_gbs, "d2h_gbs_alone": d2h_gbs}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on the host cores: one whole step at the metric's
        # tolerance, timed; then (untimed) the same step solved to 1e-13, the
        # reference each GPU form's result is compared with
        t8, o8, cores = oracle_step(W, 1e-8)
        it8 = int(o8["iters"])
        del o8
        t13, o13, _ = oracle_step(W, 1e-13)
        line["cpu_baseline"] = {
            "value": 1.0 / t8, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"one whole oracle step at the full workload, timed on the wall clock "
                       f"({t8:.1f} s): marker operators, predictor, right-hand sides, FGMRES "
                       f"with the exact L^+ (DCT) to rtol 1e-8 ({it8} iterations, all run), "
                       f"force recovery, update, diagnostics; scipy.fft workers = {cores}, "
                       f"sparse products single-threaded"),
            "cpu": cpu_model()}
        line["oracle_error"] = {
            "reference": (f"oracle step solved to rtol 1e-13 ({int(o13['iters'])} FGMRES "
                          f"iterations, {t13:.1f} s); errors of each GPU form's step result "
                          f"(rtol 1e-8): relative 2-norm, and the largest element difference "
                          f"over the largest oracle element, over all and on the shell "
                          f"cells/faces"),
            **{name: oracle_errors(o13, r) for name, r in results.items()}}
        del o13
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def adjoint_bench(s, W, X, U, f, out, zf, zc, zk, timed, K):
    """Adjoint of one step: on the headline workload (mixed form, rtol 1e-8,
    cotangent of drag_z + torque_z of body 0) and on the 128^3 oscillating
    sphere with 16000 markers (FP64 form, rtol 1e-13, the gradient-check
    setting).  Times ibm_adjoint_step after its forward step."""
    import numpy as np
    import torch
    from paper_2501_15314_gb300 import _lib
    from paper_2501_15314_gb300 import workloads as wl
    from paper_2501_15314_gb300.api import IBMSolver

    def one(solver, Xd, Ud, fd, o_u, o_F, z_k, bid, centers, kw):
        solver.set_markers(Xd)
        solver.step(torch.zeros_like(o_u), torch.zeros_like(o_u),
                    torch.zeros(solver.m, dtype=torch.float64, device="cuda"), z_k, Ud, fd,
                    out=dict(u=o_u, p=torch.empty(solver.m, dtype=torch.float64, device="cuda"),
                             F=o_F), **kw)
        loads = solver.body_forces(o_F, Xd, bid, centers)
        w = np.zeros_like(loads)
        w[0, 2] = w[0, 5] = -1.0
        F_bar, _, _ = solver.body_forces_adjoint(o_F, Xd, bid, centers, w, loads)
        solver.adjoint_step(o_u, z_k, o_F, F_bar, **kw)
        ms, st = timed(lambda: solver.adjoint_step(o_u, z_k, o_F, F_bar, **kw)[2], K)
        return ms, st[-1]

    res = {}
    kw = dict(precond_prec=_lib.IBM_PREC_FP32, rtol=1e-8)
    bid = torch.from_numpy(W.body_id.astype(np.int32)).cuda()
    ms, st = one(s, X, U, f, out["u"], out["F"], zk, bid, W.centers, kw)
    res["headline_workload_mixed"] = {"adjoint_solves_per_s": 1000.0 / ms, "ms": ms,
                                      "iters": st["iters"], "relres": st["relres_true"]}
    W4 = wl.config(4, secondary=True)
    s4 = IBMSolver(W4.n, Re=W4.Re, dt=W4.dt)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    X4, U4, f4 = dv(W4.X), dv(W4.U_gamma.ravel()), dv(W4.f_body)
    u4 = torch.empty(s4.nf, dtype=torch.float64, device="cuda")
    F4 = torch.empty(3 * W4.n_markers, dtype=torch.float64, device="cuda")
    z4 = torch.zeros_like(F4)
    bid4 = torch.from_numpy(W4.body_id.astype(np.int32)).cuda()
    kw64 = dict(precond_prec=_lib.IBM_PREC_FP64, arnoldi=_lib.IBM_ARNOLDI_FP64, rtol=1e-13,
                helm_rtol=1e-14, helm_maxit=12)
    ms4, st4 = one(s4, X4, U4, f4, u4, F4, z4, bid4, W4.centers, kw64)
    res["oscillating_sphere128_fp64"] = {
        "workload": (f"{W4.name}: 128^3, sphere r 0.15 at t = 1 of the oscillation, "
                     f"{W4.n_markers} markers, Re {W4.Re}, dt {W4.dt}, from rest"),
        "adjoint_ms": ms4, "iters": st4["iters"], "relres": st4["relres_true"]}
    s4.close()
    return res


def multistep_bench(steps=10):
    """Ten consecutive one-way steps at 128^3 (one sphere r 0.15, markers at
    spacing h, Re 100, dt 2e-3, sine-mode body force; the markers stay put;
    the stated 16000 markers, spacing h/1.86, make the scalar-C time
    integration diverge, as Table A1 of the paper reports above 1.58):
    mixed form (FP32 V-cycle, double-single Arnoldi, rtol 1e-8) against the
    FP64 form (rtol 1e-12), time per step of each and their per-step
    difference ||x_mixed - x_fp64|| / ||x_fp64|| for u, p, F (the error
    against the oracle is in the parity tests)."""
    import numpy as np
    import torch
    from paper_2501_15314_gb300 import workloads as wl
    from paper_2501_15314_gb300.api import IBMSolver
    W = wl.config(2)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    X, U, f = dv(W.X), dv(W.U_gamma.ravel()), dv(W.f_body)
    forms = {"mixed": dict(precond_prec=1, rtol=1e-8),
             "fp64": dict(precond_prec=0, arnoldi=0, rtol=1e-12, helm_rtol=1e-13,
                          helm_maxit=12)}
    runs = {}
    for name, kw in forms.items():
        s = IBMSolver(W.n, Re=W.Re, dt=W.dt)
        s.set_markers(X)
        z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")  # noqa: E731
        st = dict(u=z(s.nf), um1=z(s.nf), p=z(s.m), F=z(3 * W.n_markers))
        hist, its = [], []
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(steps):
            out, stat = s.step(st["u"], st["um1"], st["p"], st["F"], U, f, **kw)
            st["um1"], st["u"], st["p"], st["F"] = st["u"], out["u"], out["p"], out["F"]
            hist.append({k: v.clone() for k, v in out.items()})
            its.append(stat["iters"])
        e1.record(s.stream)
        torch.cuda.synchronize()
        runs[name] = (e0.elapsed_time(e1) / steps, hist, its)
        s.close()
    diff = []
    for a, b in zip(runs["mixed"][1], runs["fp64"][1]):
        diff.append({k: float(torch.linalg.norm(a[k] - b[k]) / torch.linalg.norm(b[k]))
                     for k in ("u", "p", "F")})
    return {"workload": (f"{W.name}: 128^3, sphere r 0.15, {W.n_markers} markers, Re {W.Re}, "
                         f"dt {W.dt}, {steps} consecutive steps from rest"),
            "ms_per_step_mixed": runs["mixed"][0], "ms_per_step_fp64": runs["fp64"][0],
            "iters_mixed": runs["mixed"][2], "iters_fp64": runs["fp64"][2],
            "mixed_vs_fp64_per_step": diff}


def fsi_bench(steps=200, xi=1.0, criterion=0, n=384):
    """The sedimentation workload (Sec. 3.2 two-way coupling; Model problem 3
    of Sec. 6.1.3): a sphere r = 0.08 of density ratio 1.05 released from
    rest at (0.5, 0.5, 0.7) in the 384^3 unit box, Re 50, dt 5e-4, gravity
    10 along -z, markers at spacing h; FP32 V-cycle, inner Schur solves to
    1e-2, relaxation xi, corrections until ||F'||_1/||F||_1 < 1e-3.  `steps`
    consecutive steps from release, each timed with CUDA events (every step
    synchronises for its correction count).  criterion: the norm of the
    stopping test, on the marker force densities (0, as Eq.
    (convergence_criterion) is written) or on the spread ones (1)."""
    import numpy as np
    import torch
    from paper_2501_15314_gb300 import workloads as wl
    from paper_2501_15314_gb300.api import IBMSolver, RigidSpheres
    r, th, dt = 0.08, 1.05, 5e-4
    nm = wl.markers_for_spacing(r, 1.0 / n)
    L0 = torch.from_numpy(wl.fibonacci_sphere(nm, r, [0.0, 0.0, 0.0])).cuda()
    bid = torch.zeros(nm, dtype=torch.int32, device="cuda")
    sp = RigidSpheres([r], [th], [(0.5, 0.5, 0.7)])
    s = IBMSolver(n, Re=50.0, dt=dt)
    z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")  # noqa: E731
    st_ = dict(u=z(s.nf), um1=z(s.nf), p=z(s.m), F=z(3 * nm))
    outs = [dict(X=z(3 * nm), u=z(s.nf), p=z(s.m), F=z(3 * nm)) for _ in range(3)]
    ms, inner, fg, usz = [], [], [], []
    torch.cuda.synchronize()
    for k in range(steps):
        o = outs[k % 3]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        out, st = s.fsi_step(sp, L0, bid, st_["u"], st_["um1"], st_["p"], st_["F"], None,
                             out=o, gravity=(0.0, 0.0, -10.0), xi=xi, tol=1e-3, max_inner=200,
                             rtol=1e-2, criterion=criterion, raise_on_error=False)
        e1.record(s.stream)
        torch.cuda.synchronize()
        st_["um1"], st_["u"], st_["p"], st_["F"] = st_["u"], out["u"], out["p"], out["F"]
        ms.append(e0.elapsed_time(e1))
        inner.append(int(st["inner"]))
        fg.append(int(st["fgmres_iters"]))
        usz.append(float(sp.get("us")[0, 2]))
    s.close()
    last = slice(steps // 2, steps)
    return {"workload": (f"sediment{n}: {n}^3, sphere r {r} density ratio {th}, Re 50, dt {dt}, "
                         f"g 10, {nm} markers, {steps} steps from release, xi {xi}, stopping "
                         f"test on the {'spread' if criterion else 'marker'} force densities"),
            "steps": steps, "wall_s": sum(ms) / 1e3, "ms_per_step": sum(ms) / steps,
            "ms_per_step_second_half": float(np.mean(ms[last])),
            "corrections_mean": float(np.mean(inner)),
            "corrections_second_half_mean": float(np.mean(inner[last])),
            "corrections_max": int(max(inner)),
            "corrections_per_step": inner, "fgmres_iters_per_step": fg,
            "ms_per_step_each": [round(v, 2) for v in ms],
            "u_s_z_every_10": usz[9::10]}


def porous_bench(timed, K):
    """The headline step (mixed form, rtol 1e-8) on a second geometry: the
    porous spheres of Sec. 6.1.2 (7 and 14 sub-spheres of Table 1, markers at
    spacing h) at 256^3."""
    import numpy as np
    import torch
    from paper_2501_15314_gb300 import _lib
    from paper_2501_15314_gb300 import workloads as wl
    from paper_2501_15314_gb300.api import IBMSolver
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    res = {}
    for k in (7, 14):
        Wp = wl.porous_sphere(256, k)
        sp = IBMSolver(Wp.n, Re=Wp.Re, dt=Wp.dt)
        X, U, f = dv(Wp.X), dv(Wp.U_gamma.ravel()), dv(Wp.f_body)
        zf = torch.zeros(sp.nf, dtype=torch.float64, device="cuda")
        zc = torch.zeros(sp.m, dtype=torch.float64, device="cuda")
        zk = torch.zeros(3 * Wp.n_markers, dtype=torch.float64, device="cuda")
        o = dict(u=torch.empty_like(zf), p=torch.empty_like(zc), F=torch.empty_like(zk))

        def one():
            sp.set_markers(X)
            return sp.step(zf, zf, zc, zk, U, f, out=o, precond_prec=_lib.IBM_PREC_FP32,
                           rtol=1e-8)[1]
        one()
        ms, st = timed(one, K)
        res[f"{k}_subspheres"] = {
            "workload": (f"{Wp.name}: 256^3, {k} sub-spheres r {Wp.radii[0]:.4f} in a bounding "
                         f"sphere D 0.3 at t = 1 of the oscillation, {Wp.n_markers} markers"),
            "steps_per_s": 1000.0 / ms, "ms": ms, "iters": st[-1]["iters"],
            "relres": st[-1]["relres_true"]}
        sp.close()
    return res


def cmode_bench(timed, K):
    """The three treatments of C = R^T R on one Schur solve of the step's form
    at 128^3 (one sphere r = 0.15, markers at spacing h: C is well enough
    conditioned for the inner conjugate gradients), rtol 1e-8, FP32 V-cycle
    with the double-single Arnoldi process."""
    import numpy as np
    import torch
    from paper_2501_15314_gb300 import _lib
    from paper_2501_15314_gb300 import workloads as wl
    from paper_2501_15314_gb300.api import IBMSolver
    W2 = wl.config(2)
    s2 = IBMSolver(W2.n, Re=W2.Re, dt=W2.dt)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    s2.set_markers(dv(W2.X))
    f2 = dv(W2.f_body)
    a = 1.5 / W2.dt
    rhs_F = a * (s2.interp(f2) - dv(W2.U_gamma.ravel()))
    b = a * s2.gradient_t(f2) + 2.0 * s2.gradient_t(s2.spread(rhs_F))
    res = {"workload": (f"{W2.name}: 128^3, one sphere r 0.15, {W2.n_markers} markers "
                        f"(spacing h), solve of the step's form, rtol 1e-8")}
    for name, mode in (("scalar", _lib.IBM_CMODE_SCALAR), ("exact", _lib.IBM_CMODE_EXACT),
                       ("consistent", _lib.IBM_CMODE_CONSISTENT)):
        kw = dict(precond_prec=_lib.IBM_PREC_FP32, rtol=1e-8, maxit=400, restart=60,
                  c_mode=mode, c_rtol=1e-12)
        if mode == _lib.IBM_CMODE_SCALAR:
            s2.solve_schur(b, raise_on_error=False, **kw)
        # the C modes run for seconds: one timed solve, after the scalar one
        # has set up the workspace
        k = K if mode == _lib.IBM_CMODE_SCALAR else 1
        ms, st = timed(lambda: s2.solve_schur(b, raise_on_error=False, **kw)[1], k)
        res[name] = {"solves_per_s": 1000.0 / ms, "ms": ms, "iters": st[-1]["iters"],
                     "relres": st[-1]["relres_true"], "inner_cg_iters": st[-1]["c_iters"]}
    s2.close()
    return res


def run_profile_step(args):
    """One warm-up step, then one step inside cudaProfilerStart/Stop."""
    import numpy as np
    import torch
    from paper_2501_15314_gb300 import _lib
    from paper_2501_15314_gb300 import workloads as wl
    from paper_2501_15314_gb300.api import IBMSolver
    W = wl.config(args.config, secondary=True)
    if args.grid and args.grid != W.n:
        # the same bodies and marker count on another grid (smaller captures)
        W = wl.spheres_workload(f"{W.name}_at{args.grid}", args.grid, W.Re, W.dt, W.centers,
                                W.radii, W.n_markers, args.config)
    s = IBMSolver(W.n, Re=W.Re, dt=W.dt)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    X, U, f = dev(W.X), dev(W.U_gamma.ravel()), dev(W.f_body)
    zf = torch.zeros(s.nf, dtype=torch.float64, device="cuda")
    zc = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    zk = torch.zeros(3 * W.n_markers, dtype=torch.float64, device="cuda")
    prec = _lib.IBM_PREC_FP64 if args.fp64 else _lib.IBM_PREC_FP32
    arn = _lib.IBM_ARNOLDI_FP64 if args.fp64 else _lib.IBM_ARNOLDI_FP32

    def step():
        s.set_markers(X)
        return s.step(zf, zf, zc, zk, U, f, precond_prec=prec, arnoldi=arn, rtol=1e-8,
                      restart=args.restart)[1]

    step()
    torch.cuda.synchronize()
    l0 = s.lib.ibm_kernel_launches()
    torch.cuda.cudart().cudaProfilerStart()
    t = time.perf_counter()
    st = step()
    torch.cuda.synchronize()
    t = time.perf_counter() - t
    torch.cuda.cudart().cudaProfilerStop()
    print(json.dumps({"profile_step": W.name, "ms": 1e3 * t, "iters": st["iters"],
                      "launches": int(s.lib.ibm_kernel_launches() - l0)}), flush=True)
    s.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-step", action="store_true")
    ap.add_argument("--fp64", action="store_true", help="profile the plain FP64 form")
    ap.add_argument("--grid", type=int, default=0, help="profile step: grid size override")
    ap.add_argument("--restart", type=int, default=40, help="profile step: FGMRES restart")
    ap.add_argument("--fsi-steps", type=int, default=200,
                    help="two-way sedimentation steps at 384^3 (0: skip the record)")
    ap.add_argument("--fsi-xi", type=float, default=1.0, help="two-way relaxation factor")
    args = ap.parse_args()
    if args.profile_step:
        return run_profile_step(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
