"""Benchmark: Euler RHS cell-updates/s of the regularized WENO-IS solver on GB300.

Workload: the double Mach reflection of Sec. 4.5 of the paper on a 2048 x 512
grid (LLF splitting, hybrid on, RK3 at CFL 0.5), synthetic initial data as the
paper defines them, advanced on the GPU from t = 0 to t = 0.05 (untimed) so
that the Mach stem, slip line and reflected shocks are present.  A step is one
full RK3 step (CFL max-reduction, three stages of ghost cells + x/y sweeps
with the RK combination fused); one step is 3 cell-updates per cell.

`value` is the FP64 path.  The FP32 and mixed paths are timed on the same
state and reported with their L1/Linf density error against the FP64 path
after the same number of steps.  L2 is flushed (256 MiB write) between timed
steps.  `--impl reference` times the FP64 CPU oracle (the reference arm of
this project) on the same developed state.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Euler RHS cell-updates/s on 1 GB300 (FP64 vs FP32), % roofline, L1 err vs FP64"
UNIT = "cell-updates/s"
NX, NY = 2048, 512
T_DEVELOP = 0.05

# Algorithmic flops (add/sub, mul, div, sqrt each count one) of the method as
# written in the paper, from the operation-counting instantiation of the CPU
# oracle: per cell (primitives + physical flux of one sweep direction), per
# linear-upwind face and per WENO face, by dimension.  The flux divergence
# adds 2 flops per variable per cell.
ALG_FLOPS = {1: (18, 158, 1139), 2: (22, 221, 1625), 3: (26, 292, 2167)}
# The same counts without the operations the oracle folds between known
# constants (e.g. 13/12) and without products, sums and quotients with
# structural 0 or +-1 entries (of the eigenvector matrices, E_2 = E_3 = 0).
ALG_FLOPS_ESSENTIAL = {1: (17, 151, 1060), 2: (21, 203, 1451), 3: (25, 255, 1842)}
# Of a cell's operations, those of its physical flux and eigenvalues along
# the sweep direction (F: dim products, the pressure sum, E + p and its
# product; lambda: u_n - c, u_n + c).  The rest (velocity, |u|^2, p, c, H)
# does not depend on the direction: the FP64 library computes it in the first
# sweep of a stage and the other directions read it, so a reading sweep is
# credited with these per cell instead of the whole cell count.
ALG_FLOPS_CELL_DIR = {1: 6, 2: 7, 3: 8}
FP64_FLOP_PER_CLK_SM = 4      # 2 DFMA lanes per SM per clock on GB300
FP32_FLOP_PER_CLK_SM = 256    # 128 FFMA lanes per SM per clock


# sources of the sweep kernel that the committed ncu figures describe
SWEEP_SOURCES = ("weno_device.cuh", "weno_kernels.cuh", "weno_launch.cuh", "weno_f64.cu", "weno_f32.cu")


def csrc_digest() -> str:
    """Digest of the sweep kernel's sources (profiles/traffic.json is used only
    while it matches)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1908_02464_gb300", "csrc")
    for f in SWEEP_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def nsm_sm_max(torch) -> float:
    """SM count x maximum SM clock in Hz (the clock from MEASURED_PEAKS.json)."""
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return nsm * float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = str(index)
        try:
            import torch
            u = str(torch.cuda.get_device_properties(index).uuid)
            self.index = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", self.index], stdout=self.out, stderr=subprocess.DEVNULL)
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
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank timing over all ranks (the slowest rank sets the
    aggregate rate); the identity on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(count: int, rank: int, world: int):
    """Instances of a batch of independent problems owned by one rank."""
    return list(range(rank, count, world))


def reads_prims(precision: str, dim: int, d: int) -> bool:
    """Whether the library's sweep along d reads the stage's cell primitives
    (FP64 grids of two or three dimensions: every direction but the first
    swept, which is the last one)."""
    return precision == "fp64" and dim > 1 and d != dim - 1


def sweep_flops(dim: int, n, weno_faces: int, d: int, table=None, prims_read: bool = False) -> float:
    fc, fu, fw = (table or ALG_FLOPS)[dim]
    if prims_read:
        fc = ALG_FLOPS_CELL_DIR[dim]
    cells = float(np.prod(n))
    faces = cells / n[d] * (n[d] + 1)
    return cells * (fc + 2 * (dim + 2)) + faces * fu + weno_faces * (fw - fu)


def workload_config(ws: int) -> dict:
    """The timed workload, identical for both arms (no measured values)."""
    return {"workload": f"double Mach reflection {NX}x{NY} (Sec. 4.5), FP64, state developed from t=0 to "
                        f"t={T_DEVELOP} (untimed), LLF splitting, hybrid on, TVD RK3 CFL 0.5",
            "grid": [NX, NY], "cells": NX * NY, "precision": "fp64", "t_start": T_DEVELOP,
            "parallelism": f"replicas x{ws}", "l2": "flushed between timed steps (256 MiB write)"}


def developed_state(stream=None):
    """The benchmark's input: the double Mach reflection advanced from its
    initial condition to t = T_DEVELOP by the library (FP64, untimed).
    Returns the solver holding it and the state as a device tensor."""
    from paper_1908_02464_gb300 import problems as P
    from paper_1908_02464_gb300 import weno
    prob, U0 = P.double_mach(NX, NY)
    s = weno.Solver(prob, "fp64", stream=stream)
    s.set_state(U0)
    s.advance(T_DEVELOP)
    Udev, t_dev = s.get_state(device=True)
    return s, Udev, t_dev


# ---------------------------------------------------------------- our arm
def run_ours(args) -> dict:
    import torch
    from paper_1908_02464_gb300 import problems as P
    from paper_1908_02464_gb300 import weno

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    cells = NX * NY
    prob, U0 = P.double_mach(NX, NY)
    stream = torch.cuda.current_stream()

    clocks = ClockSampler(dev)
    clocks.start()
    # developed state (untimed)
    s64, Udev, t_dev = developed_state(stream)
    Udev_host = np.ascontiguousarray(Udev.cpu().numpy())
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device="cuda")   # 256 MiB

    tiles = {}

    def timed(solver, K, W):
        solver.set_state(Udev, t_dev)
        tiles[solver.precision] = solver.autotune(3)
        solver.enqueue_steps(1.0, W)
        torch.cuda.synchronize()
        solver.weno_faces(reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(f"timed_{solver.precision}")
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            solver.enqueue_steps(1.0, 1)
            e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = [a.elapsed_time(b) for a, b in ev]
        wf = solver.weno_faces()
        return ms, wf

    ms64, wf64 = timed(s64, args.steps, args.warmup)
    tot = max_over_ranks(sum(ms64), device="cuda")
    value = ws * 3.0 * cells * args.steps / (tot * 1e-3)
    U64, t64 = s64.get_state()
    n_faces_step = 3 * ((NX + 1) * NY + NX * (NY + 1))
    weno_frac = wf64 / (n_faces_step * args.steps)

    # dominant kernel: per-direction sweep times on the state after the timed steps
    torch.cuda.nvtx.range_push("sweeps_fp64")
    ms_dir, wf_dir = s64.time_sweeps(reps=args.sweep_reps, flush=flush)
    torch.cuda.nvtx.range_pop()
    dom = int(np.argmax(ms_dir))
    fl = sweep_flops(2, [NX, NY], wf_dir[dom], dom, prims_read=reads_prims("fp64", 2, dom))
    fl_ess = sweep_flops(2, [NX, NY], wf_dir[dom], dom, ALG_FLOPS_ESSENTIAL, prims_read=reads_prims("fp64", 2, dom))
    achieved = fl / (ms_dir[dom] * 1e-3)
    peak64 = nsm * FP64_FLOP_PER_CLK_SM * sm_max * 1e6
    frac_dir = [sweep_flops(2, [NX, NY], wf_dir[d], d, prims_read=reads_prims("fp64", 2, d)) / (ms_dir[d] * 1e-3)
                / peak64 for d in range(2)]
    # the whole step: the sweeps' algorithmic flops of three stages (the WENO
    # faces counted by the kernels in the timed steps) over the step's event
    # time, which also holds the CFL reduction and the bookkeeping kernels
    fc_full, fu, fw = ALG_FLOPS[2]
    step_fl = 0.0
    for d in range(2):
        fcd = ALG_FLOPS_CELL_DIR[2] if reads_prims("fp64", 2, d) else fc_full
        nf = (NX + (d == 0)) * (NY + (d == 1))
        step_fl += 3.0 * (cells * (fcd + 2 * 4) + nf * fu)
    step_fl += wf64 / args.steps * (fw - fu)
    micro64, _ = weno.weno_measure_fma_peak(0)
    traffic = None
    pipe_ncu = None
    executed = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        with open(tp) as f:
            tj = json.load(f)
        if tj.get("csrc_digest") == csrc_digest():
            traffic = tj.get("fp64", {}).get(f"sweep_dir{dom}")
            pipe_ncu = tj.get("fp64", {}).get("pipe_fp64_pct_active", {}).get(f"sweep_dir{dom}")
            mix = tj.get("fp64", {}).get("thread_inst", {}).get(f"sweep_dir{dom}")
            if mix:
                # executed FP64 flops of the captured launch (DFMA = 2) over the event time
                ex = mix["dadd"] + mix["dmul"] + 2.0 * mix["dfma"]
                executed = {"flops_per_launch": ex, "achieved": ex / (ms_dir[dom] * 1e-3) / 1e12,
                            "frac": ex / (ms_dir[dom] * 1e-3) / peak64,
                            "source": "ncu thread-instruction counts (DADD + DMUL + 2 DFMA), profiles/traffic.json"}
    hbm_peak = None
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        with open(mp) as f:
            hbm_peak = json.load(f).get("hbm_gbs")
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak64 / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak64, "traffic": traffic,
                "achieved_essential": fl_ess / (ms_dir[dom] * 1e-3) / 1e12,
                "frac_essential": fl_ess / (ms_dir[dom] * 1e-3) / peak64,
                "alg_flops_essential_per_launch": fl_ess, "executed": executed,
                "kernel": f"k_sweep<double,2,{dom}> ({'x' if dom == 0 else 'y'}-sweep)",
                "kernel_ms": ms_dir[dom], "alg_flops_per_launch": fl, "weno_faces_per_launch": int(wf_dir[dom]),
                "frac_per_dir": frac_dir,
                "step": {"alg_flops": step_fl, "ms": tot / args.steps,
                         "frac": step_fl / (tot / args.steps * 1e-3) / peak64},
                "cell_flops_credited": {"first_sweep": fc_full, "reading_sweeps": ALG_FLOPS_CELL_DIR[2],
                                        "note": "the y-sweep computes and stores the cell primitives, the x-sweep "
                                                "reads them and is credited with the direction-dependent "
                                                "cell operations only"},
                "peak_source": f"derived: {nsm} SMs x {FP64_FLOP_PER_CLK_SM} FP64 flop/clk x {sm_max:.0f} MHz",
                "peak_fma_microbenchmark": micro64 / 1e12, "sweep_ms_per_dir": ms_dir,
                "sweep_share_of_step": 3 * sum(ms_dir) / (tot / args.steps),
                "fp64_pipe_pct_active_ncu": pipe_ncu,
                "dram_gbs": None if traffic is None else traffic / (ms_dir[dom] * 1e-3) / 1e9,
                "dram_frac_of_measured_hbm": (None if traffic is None or not hbm_peak
                                              else traffic / (ms_dir[dom] * 1e-3) / 1e9 / hbm_peak)}

    # reduced-precision paths on the same state
    extra = {}
    flags64 = None
    if not args.fp64_only:
        for prec in ("fp32", "mixed"):
            sp = weno.Solver(prob, prec, stream=stream)
            msp, wfp = timed(sp, args.steps, args.warmup)
            Up, tp_ = sp.get_state()
            totp = sum(msp)
            d = np.abs(Up[0].astype(np.float64) - U64[0])
            torch.cuda.nvtx.range_push(f"sweeps_{prec}")
            ms_d, wf_d = sp.time_sweeps(reps=5, flush=flush)
            torch.cuda.nvtx.range_pop()
            # hybrid-switch decisions against FP64 on the same float-rounded state
            # (arithmetic only; storage rounding is the same on both sides)
            Uf = np.ascontiguousarray(U64.astype(np.float32))
            fl_p = sp.face_flags(torch.from_numpy(Uf).cuda(), t64).cpu().numpy()
            if flags64 is None:
                flags64 = s64.face_flags(torch.from_numpy(Uf.astype(np.float64)).cuda(), t64).cpu().numpy()
            dd = int(np.argmax(ms_d))
            flp = sweep_flops(2, [NX, NY], wf_d[dd], dd)
            peak32 = nsm * FP32_FLOP_PER_CLK_SM * sm_max * 1e6
            extra[prec] = {"value": ws * 3.0 * cells * args.steps / (totp * 1e-3), "ms_per_step": totp / args.steps,
                           "l1_rho_vs_fp64": float(np.mean(d)), "linf_rho_vs_fp64": float(np.max(d)),
                           "weno_face_fraction": wfp / (n_faces_step * args.steps),
                           "hybrid_flags_differing_from_fp64_same_data": int(np.sum(fl_p != flags64)),
                           "faces": int(flags64.size),
                           "t_after": tp_, "t_fp64_after": t64,
                           "roofline": {"bound": "alu", "achieved": flp / (ms_d[dd] * 1e-3) / 1e12,
                                        "peak": peak32 / 1e12, "unit": "TFLOP/s",
                                        "frac": flp / (ms_d[dd] * 1e-3) / peak32,
                                        "kernel_ms": ms_d[dd], "sweep_ms_per_dir": ms_d}}
            sp.close()

    clk = clocks.stop()
    clk["window"] = "development run + all timed regions (FP64, FP32, mixed)"

    # end to end through the public API with pinned host buffers
    e2e_steps = min(args.steps, 10)
    Uh = torch.from_numpy(np.ascontiguousarray(U64)).pin_memory()
    Uo = torch.empty_like(Uh).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tcur = t64
    for _ in range(e2e_steps):
        s64.set_state(Uh, tcur)
        s64.step(1.0)
        tcur = weno.weno_get_state(s64.ctx, Uo)
        Uh, Uo = Uo, Uh
    el = time.perf_counter() - t0
    e2e = {"value": ws * 3.0 * cells * e2e_steps / el, "unit": UNIT, "h2d_bytes_per_step": Uh.numel() * 8,
           "d2h_bytes_per_step": Uh.numel() * 8, "steps": e2e_steps,
           "api": "weno_set_state(host) + weno_step + weno_get_state(host)"}
    s64.close()

    batch = None if args.no_batch else batched_riemann(args)
    batch2 = None if args.no_batch else batched_2d(args)
    vortex = None if args.no_vortex else vortex3d_rhs_vjp(args)
    jet = None if args.no_jet else mach2000_jet_run(args)
    shu = None if args.no_shu else shu_osher_precisions(args)
    thr = None if args.no_shu else threshold_study(args)

    launches_per_step = 3 + 3 * 2 + 1   # cfl, dt, post, 3 stages x 2 sweeps, set_tend
    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": tot / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(ws),
           "workload_stats": {"weno_face_fraction": weno_frac, "t_start": t_dev, "t_after": t64,
                              "tiles_autotuned": tiles},
           "roofline": roofline, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
           "clocks": clk, "ms_per_step_all": ms64}
    res.update(extra)
    if batch is not None:
        res["batched_riemann"] = batch
    if batch2 is not None:
        res["batched_2d"] = batch2
    if vortex is not None:
        res["vortex3d_256"] = vortex
    if jet is not None:
        res["mach2000_jet"] = jet
    if shu is not None:
        res["shu_osher_400"] = shu
    if thr is not None:
        res["threshold_study_shu_osher_400"] = thr
    if rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args, Udev_host, t_dev)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return res if rank == 0 else None


def batched_riemann(args) -> dict:
    """4096 random 1D Riemann problems (N ~ U[100, 4000]) solved to their own
    end times by one persistent, graph-replayed launch per precision."""
    import torch
    from paper_1908_02464_gb300 import problems as P
    from paper_1908_02464_gb300 import weno
    params, redraws = P.riemann_batch_params(args.batch_count, seed=20190807)
    states = [P.riemann_instance(params, i)[1] for i in range(args.batch_count)]
    out = {"instances": args.batch_count, "cells": int(params["N"].sum()), "redraws": redraws,
           "workload": "random Riemann problems on [0,1], rho and p log-uniform in [0.01, 10], u in [-2, 2], "
                       "N ~ U[100, 4000], t_end = 0.2 / max(|u|+c), seed 20190807, transmissive"}
    ref = None
    for prec in ("fp64", "fp32", "mixed"):
        b = weno.Batch(params["N"], 0.0, 1.0, params["t_end"], prec)
        U0 = b.pack(states)
        U = U0.clone()
        choice = b.autotune(U, trial_steps=8)
        b.weno_faces(reset=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run(U)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st, steps, t = b.results()
        wf = b.weno_faces()
        cu = 3.0 * float(np.sum(params["N"] * steps))
        # algorithmic flops of the sweeps (oracle operation counts, 1D): per
        # stage N cells, N + 1 faces, and the counted WENO faces
        fc, fu, fw = ALG_FLOPS[1]
        stage_units = 3.0 * steps.astype(np.float64)
        fl = float(np.sum(stage_units * (params["N"] * (fc + 2 * 3) + (params["N"] + 1) * fu))) + wf * (fw - fu)
        peak = nsm_sm_max(torch) * (FP64_FLOP_PER_CLK_SM if prec == "fp64" else FP32_FLOP_PER_CLK_SM)
        entry = {"value": cu / (ms * 1e-3), "unit": UNIT, "seconds": ms * 1e-3, "cell_updates": cu,
                 "nonphysical_instances": int(np.sum(st != 0)), "tile_variant": choice[0], "ctas": choice[1],
                 "steps_total": int(steps.sum()), "weno_faces": int(wf),
                 "weno_face_fraction": wf / float(np.sum(stage_units * (params["N"] + 1))),
                 "roofline": {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12, "peak": peak / 1e12,
                              "unit": "TFLOP/s", "frac": fl / (ms * 1e-3) / peak,
                              "note": "algorithmic sweep flops (oracle counts) of the whole persistent launch "
                                      "over its event time; CFL reductions not counted"}}
        res = b.unpack(U)
        if prec == "fp64":
            ref = res
        else:
            ok = [i for i in range(b.count) if st[i] == 0]
            l1 = [float(np.mean(np.abs(res[i][0] - ref[i][0]))) for i in ok]
            entry["l1_rho_vs_fp64_mean"] = float(np.mean(l1))
            entry["l1_rho_vs_fp64_max"] = float(np.max(l1))
        out[prec] = entry
        b.close()
    return out


def batched_2d(args) -> dict:
    """4096 random 2D cylindrical explosions and implosions in boxes of
    16..64 x 16..64 cells, each solved to its own end time by one persistent,
    graph-replayed launch per precision (autotuned tiles and residency)."""
    import torch
    from paper_1908_02464_gb300 import problems as P
    from paper_1908_02464_gb300 import weno
    params, redraws = P.explosion_batch_params(args.batch_count, seed=20190808)
    states = [P.explosion_instance(params, i)[1] for i in range(args.batch_count)]
    NX, NY = params["NX"], params["NY"]
    cells = NX * NY
    out = {"instances": args.batch_count, "cells": int(cells.sum()), "redraws": redraws,
           "workload": "disc of radius U[0.15, 0.35] min(Lx, Ly) at rest in gas at rest, rho and p log-uniform in "
                       "[0.1, 10] inside and out (density ratio <= 20), NX, NY ~ U{16..64}, square cells of 1/64, "
                       "t_end = 0.2 min(Lx, Ly) / max c, seed 20190808, transmissive"}
    ref = None
    hi = np.stack([NX * params["h"], NY * params["h"]], axis=1)
    for prec in ("fp64", "fp32", "mixed"):
        b = weno.Batch2D(NX, NY, (0.0, 0.0), hi, params["t_end"], prec)
        U = b.pack(states)
        choice = b.autotune(U, trial_steps=8)
        b.weno_faces(reset=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run(U)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st, steps, t = b.results()
        wf = b.weno_faces()
        stage_units = 3.0 * steps.astype(np.float64)
        cu = float(np.sum(cells * stage_units))
        # algorithmic flops of the two sweeps per stage (oracle operation
        # counts, 2D): cells x 2 directions, x and y faces, counted WENO faces
        faces = (NX + 1) * NY + NX * (NY + 1)
        fc, fu, fw = ALG_FLOPS[2]
        fl = float(np.sum(stage_units * (2 * cells * (fc + 2 * 4) + faces * fu))) + wf * (fw - fu)
        peak = nsm_sm_max(torch) * (FP64_FLOP_PER_CLK_SM if prec == "fp64" else FP32_FLOP_PER_CLK_SM)
        entry = {"value": cu / (ms * 1e-3), "unit": UNIT, "seconds": ms * 1e-3, "cell_updates": cu,
                 "nonphysical_instances": int(np.sum(st != 0)), "tile_variant": choice[0], "ctas": choice[1],
                 "steps_total": int(steps.sum()), "weno_faces": int(wf),
                 "weno_face_fraction": wf / float(np.sum(stage_units * faces)),
                 "roofline": {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12, "peak": peak / 1e12,
                              "unit": "TFLOP/s", "frac": fl / (ms * 1e-3) / peak,
                              "note": "algorithmic sweep flops (oracle counts) of the whole persistent launch "
                                      "over its event time; CFL reductions not counted"}}
        res = b.unpack(U)
        if prec == "fp64":
            ref = res
        else:
            ok = [i for i in range(b.count) if st[i] == 0]
            l1 = [float(np.mean(np.abs(res[i][0] - ref[i][0]))) for i in ok]
            entry["l1_rho_vs_fp64_mean"] = float(np.mean(l1))
            entry["l1_rho_vs_fp64_max"] = float(np.max(l1))
        out[prec] = entry
        b.close()
    return out


def shu_osher_precisions(args) -> dict:
    """Shock / entropy-wave interaction (Sec. 4.4 shifted to [-5, 5]) at 400
    cells to t = 1.8 in FP64, FP32 and mixed: L1 / Linf error of density
    against the oracle's 3200-cell solution stored in tests/golden, and the
    wall time of the run (launch-bound at this size)."""
    import torch
    from paper_1908_02464_gb300 import problems as P
    from paper_1908_02464_gb300 import weno
    path = os.path.join(ROOT, "tests", "golden", "shu_osher_rho_ref400.txt")
    ref = np.array([float(l) for l in open(path) if not l.startswith("#")])
    prob, U = P.shu_osher(400)
    out = {"cells": 400, "t_end": prob["t_end"],
           "reference": "FP64 oracle on 3200 cells averaged onto 400 (tests/golden/shu_osher_rho_ref400.txt)"}
    for prec in ("fp64", "fp32", "mixed"):
        s = weno.Solver(prob, prec)
        s.set_state(U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = s.advance(prob["t_end"])
        wall = time.perf_counter() - t0
        V, _ = s.get_state()
        s.close()
        r = V[0].astype(np.float64)
        out[prec] = {"l1_rho": float(np.mean(np.abs(r - ref))), "linf_rho": float(np.max(np.abs(r - ref))),
                     "steps": k, "wall_s": wall, "cell_updates_per_s": 3.0 * 400 * k / wall}
    return out


def threshold_study(args) -> dict:
    """The switch threshold eps_h = C (dx / L)^3 of Sec. 3 against accuracy:
    Shu-Osher at 400 cells to t = 1.8 in FP64 for several characteristic
    lengths L, with the per-face and the per-field hybrid and with the hybrid
    off.  Per run: the fraction of faces that took the WENO flux (the
    solver's own counter), L1 / Linf of density against the oracle's
    3200-cell solution, steps and wall time."""
    import torch
    from paper_1908_02464_gb300 import problems as P
    from paper_1908_02464_gb300 import weno
    path = os.path.join(ROOT, "tests", "golden", "shu_osher_rho_ref400.txt")
    ref = np.array([float(l) for l in open(path) if not l.startswith("#")])
    runs = [(0, 1.0)] + [(h, L) for h in (1, 2) for L in (0.25, 0.5, 1.0, 2.0, 4.0, 8.0)]
    out = {"cells": 400, "t_end": 1.8, "precision": "fp64", "C_thr": 1.0, "alpha_thr": 3,
           "hybrid_modes": {"0": "off (WENO everywhere)", "1": "per face", "2": "per field"}, "runs": []}
    for hybrid, L in runs:
        prob, U = P.shu_osher(400)
        prob["hybrid"] = hybrid
        prob["L_char"] = L
        s = weno.Solver(prob, "fp64")
        s.set_state(U)
        s.weno_faces(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = s.advance(prob["t_end"])
        wall = time.perf_counter() - t0
        wf = s.weno_faces()
        V, _ = s.get_state()
        s.close()
        r = V[0].astype(np.float64)
        out["runs"].append({"hybrid": hybrid, "L_char": L, "steps": k,
                            "weno_face_fraction": wf / (3.0 * 401 * k),
                            "l1_rho": float(np.mean(np.abs(r - ref))), "linf_rho": float(np.max(np.abs(r - ref))),
                            "wall_s": wall})
    return out


def mach2000_jet_run(args) -> dict:
    """Mach 2000 jet of Sec. 4.7 at the paper's 640 x 160 to t = 0.001 (global
    LF splitting, the workload's lambda reading), FP64 and mixed: whether the
    run finishes, its steps and wall time, and the positivity margins."""
    import torch
    from paper_1908_02464_gb300 import problems as P
    from paper_1908_02464_gb300 import weno
    prob, U = P.mach2000_jet(640, 160)
    out = {"grid": [640, 160], "t_end": prob["t_end"], "splitting": prob["splitting"],
           "c_lambda": prob["c_lambda"]}
    ref = None
    for prec in ("fp64", "mixed"):
        s = weno.Solver(prob, prec)
        s.set_state(U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            k = s.advance(prob["t_end"])
            status = "ok"
        except weno.WenoError as e:
            k, status = None, f"stopped: {e}"
        wall = time.perf_counter() - t0
        V, t = s.get_state()
        s.close()
        V = V.astype(np.float64)
        g = prob["gamma"]
        p = (g - 1.0) * (V[3] - 0.5 * (V[1] ** 2 + V[2] ** 2) / V[0])
        entry = {"status": status, "steps": k, "t": t, "wall_s": wall, "rho_min": float(V[0].min()),
                 "p_min": float(p.min())}
        if prec == "fp64":
            ref = V
        elif status == "ok" and ref is not None:
            entry["l1_rho_vs_fp64"] = float(np.mean(np.abs(V[0] - ref[0])))
        out[prec] = entry
    return out


def vortex3d_rhs_vjp(args) -> dict:
    """3D periodic vortex on 256^3: forward RHS, one RK3 step and the
    vector-Jacobian product of the RHS for a seeded N(0,1) cotangent."""
    import torch
    from paper_1908_02464_gb300 import problems as P
    from paper_1908_02464_gb300 import weno
    n = args.vortex_n
    prob, U = P.vortex3d(n)
    cells = n ** 3
    gen = torch.Generator(device="cpu").manual_seed(1)
    w = torch.randn(U.shape, generator=gen, dtype=torch.float64)
    out = {"grid": [n, n, n], "cells": cells,
           "workload": "rho=1, u=sin x cos y cos z, v=-cos x sin y cos z, w=0, p=100+(cos 2x+cos 2y)(cos 2z+2)/16 "
                       "on [0,2pi]^3 periodic; cotangent N(0,1) seed 1"}
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device="cuda")
    g64 = None
    for prec in ("fp64", "fp32"):
        s = weno.Solver(prob, prec)
        dt = torch.float64 if prec == "fp64" else torch.float32
        Ud = torch.from_numpy(U).to("cuda", dt)
        wd = w.to("cuda", dt)
        r = s.rhs(Ud)
        g = s.rhs_vjp(Ud, wd)

        def timeit(fn, reps=3):
            ts = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return min(ts)

        s.weno_faces(reset=True)
        ms_rhs = timeit(lambda: s.rhs(Ud, 0.0, out=r))
        wf = s.weno_faces() / 3.0   # per RHS evaluation (three timed evaluations)
        ms_vjp = timeit(lambda: s.rhs_vjp(Ud, wd, 0.0, out=g))
        # one more call of each inside NVTX ranges, for launch lists
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(f"rhs_{prec}")
        s.rhs(Ud, 0.0, out=r)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        torch.cuda.nvtx.range_push(f"vjp_{prec}")
        s.rhs_vjp(Ud, wd, 0.0, out=g)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        s.set_state(Ud)
        s.autotune(2)
        s.enqueue_steps(10.0, 1)
        torch.cuda.synchronize()
        ms_step = timeit(lambda: s.enqueue_steps(10.0, 1))
        # algorithmic flops of one RHS (three sweeps, oracle operation counts;
        # in FP64 the y- and x-sweeps read the primitives the z-sweep stored)
        fc, fu, fw = ALG_FLOPS[3]
        fl = 3 * (n + 1) * n * n * fu + wf * (fw - fu)
        for d in range(3):
            fl += cells * ((ALG_FLOPS_CELL_DIR[3] if reads_prims(prec, 3, d) else fc) + 2 * 5)
        peak = nsm_sm_max(torch) * (FP64_FLOP_PER_CLK_SM if prec == "fp64" else FP32_FLOP_PER_CLK_SM)
        entry = {"rhs_roofline": {"bound": "alu", "achieved": fl / (ms_rhs * 1e-3) / 1e12, "peak": peak / 1e12,
                                  "unit": "TFLOP/s", "frac": fl / (ms_rhs * 1e-3) / peak,
                                  "weno_face_fraction": wf / (3.0 * (n + 1) * n * n)},
                 "rhs_ms": ms_rhs, "rhs_cell_updates_per_s": cells / (ms_rhs * 1e-3),
                 "step_ms": ms_step, "step_cell_updates_per_s": 3 * cells / (ms_step * 1e-3),
                 "vjp_ms": ms_vjp, "vjp_cells_per_s": cells / (ms_vjp * 1e-3)}
        gh = g.double().cpu()
        if prec == "fp64":
            g64 = gh
        else:
            entry["vjp_rel_err_vs_fp64"] = float((gh - g64).abs().max() / g64.abs().max())
        out[prec] = entry
        s.close()
        del Ud, r, g
    return out


# ---------------------------------------------------------------- oracle arm
def oracle_steps(nsteps: int, U, t: float):
    """Time `nsteps` oracle RK3 steps of the benchmark grid from (U, t), in
    place.  Returns (seconds, U, t)."""
    from oracle import oracle as orc
    from paper_1908_02464_gb300 import problems as P
    prob, _ = P.double_mach(NX, NY)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        st, t, dt = orc.step(prob, U, t, 1.0)
    return time.perf_counter() - t0, U, t


def oracle_weno_fraction(U, t: float) -> float:
    """Fraction of faces on which the oracle takes the WENO flux at (U, t)."""
    from oracle import oracle as orc
    from paper_1908_02464_gb300 import problems as P
    prob, _ = P.double_mach(NX, NY)
    _, flags, _ = orc.rhs(prob, U, t, want_flags=True)
    return float(1.0 - np.mean(flags))


def host_info() -> dict:
    """Host cores and CPU model, for the CPU-baseline lines."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "hardware", "cpu model"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"host_cores": os.cpu_count(), "cpu_model": model or platform.machine()}


def oracle_worker(steps: int, state_path: str, t: float) -> None:
    """One single-threaded oracle process of the all-core baseline: loads the
    developed state, times its steps and prints the wall-clock start and end
    as one JSON line."""
    U = np.ascontiguousarray(np.load(state_path))
    t0 = time.time()
    oracle_steps(steps, U, t)
    print(json.dumps({"start": t0, "end": time.time()}), flush=True)


def cpu_all_cores(steps: int, U, t: float) -> dict:
    """The unmodified single-threaded oracle run as one process per host
    core, all at once, each on its own copy of the developed state;
    throughput = all processes' cell-updates / (last end - first start)."""
    n = os.cpu_count() or 1
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    np.save(path, U)
    try:
        cmd = [sys.executable, "-c", f"import bench; bench.oracle_worker({int(steps)}, {path!r}, {float(t)!r})"]
        procs = [subprocess.Popen(cmd, cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                 for _ in range(n)]
        spans = []
        for p in procs:
            out, _ = p.communicate()
            if p.returncode == 0 and out.strip():
                spans.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        os.unlink(path)
    if len(spans) != n:
        return {"unavailable": f"{n - len(spans)} of {n} oracle processes failed"}
    wall = max(x["end"] for x in spans) - min(x["start"] for x in spans)
    return {"value": 3.0 * NX * NY * steps * n / wall, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} concurrent single-threaded oracle processes, each {steps} FP64 RK3 steps of the "
                      f"{NX}x{NY} double Mach reflection from the developed state t = {t:.4f} ({wall:.1f} s wall)"}


def cpu_baseline(args, U, t: float) -> dict:
    """The oracle as it stands on one host core, timed on the developed state
    the GPU arm times (a bounded sample: `--cpu-steps` RK3 steps)."""
    steps = args.cpu_steps
    wf = oracle_weno_fraction(U, t)
    el, _, _ = oracle_steps(steps, U.copy(), t)
    out = {"value": 3.0 * NX * NY * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{steps} FP64 RK3 steps of the {NX}x{NY} double Mach reflection from the developed state "
                     f"t = {t:.4f} (the GPU arm's), single-threaded C++ oracle ({el:.1f} s)",
           "weno_face_fraction_at_start": wf, **host_info()}
    out["all_cores"] = cpu_all_cores(max(1, steps // 4), U, t)
    return out


def run_reference(args) -> dict | None:
    """The reference arm: the FP64 oracle timed on the same workload as the
    GPU arm.  Its input, the state developed to t = T_DEVELOP, is prepared
    by the library on the GPU, untimed: the oracle would need about 1000 steps
    of the full grid (about 12 minutes of one core) to reach it.  Without a
    GPU the arm reports itself unavailable."""
    ws, rank, local = dist_env()
    if rank != 0:
        return None
    import torch
    if not torch.cuda.is_available():
        return {"impl": "reference", "unavailable": "the timed state is prepared on the GPU and none is visible"}
    from oracle import oracle as orc
    orc.build()
    from paper_1908_02464_gb300 import build as B
    B.build()
    torch.cuda.set_device(local)
    s, Udev, t_dev = developed_state()
    U = np.ascontiguousarray(Udev.cpu().numpy())
    s.close()
    del Udev
    wf = oracle_weno_fraction(U, t_dev)
    _, U, t = oracle_steps(args.warmup, U, t_dev)
    el, U, t = oracle_steps(args.steps, U, t)
    v = 3.0 * NX * NY * args.steps / el
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(ws),
            "workload_stats": {"weno_face_fraction_at_start": wf, "t_start": t_dev, "t_after": t,
                               "input": "developed state prepared by the library on the GPU, untimed"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.warmup}+{args.steps} RK3 steps of the full grid from the developed "
                                       f"state t = {t_dev:.4f}", **host_info()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--fp64-only", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-reps", type=int, default=5)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--no-vortex", action="store_true")
    ap.add_argument("--vortex-n", type=int, default=256)
    ap.add_argument("--no-jet", action="store_true")
    ap.add_argument("--no-shu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        res = run_reference(args)
    else:
        from paper_1908_02464_gb300 import build as B
        B.build()
        from oracle import oracle as orc
        orc.build()
        res = run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
