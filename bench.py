#!/usr/bin/env python
"""Throughput of the split-explicit barotropic subcycle on GB300.

Default workload: the batched ensemble, 64 closed basins of uneven size (jittered Delaunay
meshes, log-uniform 2e4-4e5 vertices, 8.59 M vertices and 17.1 M triangles in total, M = 40,
per-basin dt), advanced together: one upload, and one sesw_advance per benchmark step for the
whole batch in the layout the autotuner picks. One benchmark step is one baroclinic step of
every basin: every row of the hot path (element pass, vertex pass, time-mean accumulation,
step epilogue) runs once per substep. Metric: vertex-substeps per second, whole job.
Other workloads: --workload channel (the 200k-vertex wind-driven channel), sphere (the
level-8 icosahedral sphere), surrogate (the learned surrogate on the sphere).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

With N > 1 (launched by torchrun) every rank advances its own copy of the
workload (independent ensemble members, no data exchange); the reported value is
the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vertex-substeps/s"
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["auto", "graph", "persistent"], default="auto")
    ap.add_argument("--persistent-form", choices=["auto", "registers", "stream", "stream-uncached"], default="auto",
                    help="channel and sphere: kernel form of the persistent mode (auto: registers unless a "
                         "patch needs 8 or more slots per thread)")
    ap.add_argument("--scheme", choices=["se", "sesm"], default="se",
                    help="se: dissipative forward-backward (Eq. 4.10); sesm: AB3-AM4 (Eqs. 4.7-4.8)")
    ap.add_argument("--visc", type=str, default=None, metavar="A_BG,C_V",
                    help="barotropic viscosity of Eq. (viscosity_BT): background (m^2/s) and flow coefficient; "
                         "'auto' picks a background at viscous number 0.2 and C_v = 1")
    ap.add_argument("--freshwater", type=float, default=0.0, metavar="AMP",
                    help="freshwater flux W of Eq. (4.5): seeded random field of this amplitude (m/s)")
    ap.add_argument("--patch-vertices", type=int, default=None,
                    help="graph-mode patch size (default 256; with --visc, one wave of the fused kernel)")
    ap.add_argument("--block-threads", type=int, default=256)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=400)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-substeps", type=int, default=4,
                    help="substeps of the channel per reference-arm step (a bounded sample)")
    ap.add_argument("--workload", choices=["channel", "sphere", "ensemble", "surrogate"], default=None,
                    help="ensemble (default): 64 basins of uneven size, batched (the headline workload); "
                         "channel: the 200k-vertex wind-driven channel (the default with --scheme sesm, --visc "
                         "or --freshwater); sphere: the global-like level-8 sphere (458,683 wet vertices); "
                         "surrogate: train and evaluate the learned surrogate on the sphere")
    ap.add_argument("--autotune", choices=["quick", "full", "none"], default="quick",
                    help="ensemble layouts timed before the run: quick (persistent forms, large-basin "
                         "layouts and one graph layout), full (every candidate), none (the layout of "
                         "--blocks-per-sm (default 1), --large-bps and --large-form)")
    ap.add_argument("--large-bps", type=int, default=0,
                    help="with --autotune none: blocks per SM of the large basins' packs (0: the same)")
    ap.add_argument("--large-form", choices=["same", "auto", "registers", "stream", "stream-uncached"],
                    default="same", help="with --autotune none: kernel form of the large basins' packs")
    ap.add_argument("--surrogate-level", type=int, default=8)
    ap.add_argument("--surrogate-traj", type=int, default=40)
    ap.add_argument("--surrogate-steps", type=int, default=50)
    ap.add_argument("--surrogate-epochs", type=int, default=3)
    ap.add_argument("--resid-tol", type=float, default=0.1)
    ap.add_argument("--ensemble-basins", type=int, default=64)
    ap.add_argument("--ensemble-scale", type=float, default=1.0)
    ap.add_argument("--sequential-steps", type=int, default=10,
                    help="ensemble: steps of the one-basin-after-another comparison (0: skip it)")
    args = ap.parse_args(argv)
    variant = args.scheme == "sesm" or bool(args.visc) or bool(args.freshwater)
    if args.workload is None:
        args.workload = "channel" if variant else "ensemble"
    elif variant and args.workload in ("ensemble", "surrogate"):
        ap.error("--scheme sesm, --visc and --freshwater run on the channel or sphere workloads")
    return args


def workload(name="channel"):
    from paper_2311_08241_gb300 import inputs as I

    if name == "sphere":
        case = I.sphere_case(level=8)
        label = ("global-like sphere: icosahedral level 8, Hilbert order, fractal bathymetry 10-6000 m with "
                 "30 % land, f = 2 Omega sin(lat), smooth random forcing, tau=1800 s, M=50")
    else:
        case = I.channel_case()
        label = ("wind-driven zonal channel 4000x2000 km, jittered Delaunay lattice, beta plane, "
                 "Gaussian ridge, tau=480 s, M=40")
    m = case.mesh
    desc = {
        "workload": label,
        "V": m.nv, "E": m.ne, "M": case.params.M, "tau_s": case.params.tau, "theta": case.params.theta,
        "nonlinear_h": case.params.nonlinear_h,
    }
    return case, desc


def algorithmic_bytes_per_substep(V, E):
    """Bytes one substep must move at minimum with FP32 state and a compensated FP32-pair mean:
    per element U r/w 16, mean pair r/w 32, corners 12, gradients 16, H0 and f 8, R 8 (92 B);
    per vertex eta r/w 8, 1/A_v 4 (12 B)."""
    return 12 * V + 92 * E


def sesm_bytes_per_substep(V, E):
    """SESM substep (k_sesm): per element three transport levels read and one written 32, mean
    pair r/w 32, corners 12, gradients 16, H0 and f 8, R 8 (108 B); per vertex four elevation
    levels read and one written 20, 1/A_v 4 (24 B)."""
    return 24 * V + 108 * E


def viscosity_bytes_per_substep(V, E):
    """What the viscosity adds to a substep (fused into k_substep, planar frames): per element the
    edge table (neighbour slots, opposite corners, rest depths, L/d, L^2/d: 64 B) and the
    start-of-step value V0 (8 B). The neighbours' U and eta are re-reads of arrays the substep
    already streams."""
    return 72 * E


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCE = {"k_persistent": ("sesw_persistent.cu", "sesw_persistent.cuh", "sesw_device.cuh"),
                 "k_persistent_sesm": ("sesw_persistent_sesm.cu", "sesw_persistent.cuh", "sesw_device.cuh"),
                 "k_persistent_stream": ("sesw_persistent_stream.cu", "sesw_persistent.cuh", "sesw_device.cuh"),
                 "k_persistent_sesm_stream": ("sesw_persistent_sesm_stream.cu", "sesw_persistent.cuh",
                                              "sesw_device.cuh")}


def kernel_source_hash(kernels=("k_persistent",)):
    """Hash of the source files of the given kernels (a profile is stale once one of them changes)."""
    if isinstance(kernels, str):
        kernels = (kernels,)
    names = []
    for k in kernels:
        for name in KERNEL_SOURCE.get(k, ("sesw_kernels.cu",)):
            if name not in names:
                names.append(name)
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2311_08241_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_figures(profile, kernels, layout=None):
    """Counters of a committed ncu summary (profiles/<profile>.md): DRAM bytes and warp instructions
    per launch (or per step, as the summary states), or None where the summary is missing or was
    taken on other kernel sources than the ones built now. With `layout`, the figures of the block
    that starts with the line "layout: <layout>" (None if the summary has no such block)."""
    p = os.path.join(ROOT, "profiles", f"{profile}.md")
    try:
        txt = open(p).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != kernel_source_hash(kernels):
        return None
    if layout is not None:
        blocks = re.split(r"(?m)^layout: ", txt)[1:]
        block = next((b for b in blocks if b.split("\n", 1)[0].strip() == layout), None)
        if block is None:
            return None
        txt = block
    out = {"profile": f"profiles/{profile}.md"}
    for key in ("dram_bytes_per_launch", "warp_instructions_per_launch", "dram_bytes_per_step",
                "warp_instructions_per_step"):
        v = re.search(key + r":\s*([0-9.eE+]+)", txt)
        if v:
            out[key] = float(v.group(1))
    return out


def profiled_traffic_for(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it matches this kernel source."""
    f = profile_figures(f"{kernel}_{workload}", (kernel,))
    return None if f is None else f.get("dram_bytes_per_launch")


def issue_peak(device_sms, sm_max_mhz):
    """Warp instructions per second the SMs can issue: 4 schedulers per SM, one warp instruction
    each per cycle, at the largest SM clock."""
    return device_sms * 4 * sm_max_mhz * 1e6


def roofline_issue(kernel, seconds, inst, dram, alg_bytes, sms, sm_max_mhz, per="launch",
                   alg_model="12 V + 92 E per substep"):
    """Roofline of an on-chip kernel: bound by instruction issue (warp instructions from the committed
    ncu capture / CUDA-event time, against the issue peak), with the DRAM rate of the same capture and
    the algorithmic-byte rate of the scope table beside it."""
    peak, src = measured_hbm_peak()
    ipk = issue_peak(sms, sm_max_mhz)
    achieved = None if inst is None else inst / seconds
    dram_gbs = None if dram is None else dram / seconds / 1e9
    return {"bound": "issue", "achieved": achieved, "peak": ipk, "unit": "warp-instructions/s",
            "frac": None if achieved is None else achieved / ipk, "traffic": dram, "traffic_per": per,
            "kernel": kernel, "seconds_per_" + per: seconds,
            "peak_from": f"{sms} SMs x 4 schedulers x {sm_max_mhz:g} MHz",
            "warp_instructions_per_" + per: inst,
            "dram": {"achieved_gbs": dram_gbs, "peak_gbs": peak, "frac": None if dram_gbs is None else dram_gbs / peak,
                     "peak_source": src},
            "algorithmic": {"bytes_per_" + per: alg_bytes, "gbs": alg_bytes / seconds / 1e9,
                            "frac_of_hbm": alg_bytes / seconds / 1e9 / peak,
                            "note": f"scope-table bytes ({alg_model}); the state stays on chip "
                                    "for the M substeps of a launch, so this is not a DRAM rate"}}


def sm_max_mhz_of(clk):
    if clk.get("sm_max_mhz"):
        return float(clk["sm_max_mhz"])
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"])
    except Exception:
        return 2070.0


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip():
                return v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model", "CPU part") and v.strip():
                    return v.strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(case, seconds, rank, W=None):
    """The FP64 oracle, as it stands, on the host cores: whole baroclinic steps until `seconds` elapse,
    all cores (the reported value), then a shorter single-thread sample for context."""
    from oracle import runner as orc

    om = orc.OracleMesh(case.mesh)
    visc = getattr(case.params, "visc", None)
    sesm = getattr(case.params, "scheme", 0) == 1
    if sesm:
        from oracle import closed

        coef = closed.sesm_params(case.params.theta / 2.0)

    def sample(budget):
        eta, U = case.eta0.copy(), case.U0.copy()
        steps = 0
        t0 = time.perf_counter()
        while True:
            if sesm:
                eta, U, _ = om.advance_sesm(case.R, case.params, coef, 1, eta, U, W=W)
            elif visc is None and W is None:
                eta, U, _, _ = om.advance(case.R, case.params, 1, eta, U)
            else:
                eta, U, _ = om.advance_ext(case.R, case.params, 1, eta, U, W=W, visc=visc)
            steps += 1
            if time.perf_counter() - t0 >= budget:
                break
        return steps, time.perf_counter() - t0

    cores = orc.set_threads(0)
    steps, dt = sample(seconds)
    orc.set_threads(1)
    steps1, dt1 = sample(max(1.0, seconds / 4))
    orc.set_threads(cores)
    om.close()
    rate = lambda n, t: case.mesh.nv * case.params.M * n / t
    return {"value": rate(steps, dt), "unit": METRIC, "cores": cores, "kind": "oracle",
            "single_thread_value": rate(steps1, dt1), "cpu_model": cpu_model(),
            "sample": f"{steps} baroclinic steps ({steps * case.params.M} substeps) of the benchmark workload "
                      f"from rest, FP64, OpenMP over {cores} threads, {dt:.1f} s wall; single thread: "
                      f"{steps1} steps in {dt1:.1f} s"}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def whole_job_value(V, M, steps, world, slowest_ms):
    """Vertex-substeps per second of all ranks together, timed by the slowest rank."""
    return world * V * M * steps / (slowest_ms * 1e-3)


def reduce_max(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def ensemble_workload(rank=0, nbasins=64, scale=1.0):
    """The batched ensemble (the scope table's batched configuration): seeded basins, per-basin dt."""
    from paper_2311_08241_gb300 import inputs as I

    cases = I.ensemble_cases(nbasins=nbasins, scale=scale, seed=20231118 + rank)
    V = sum(c.mesh.nv for c in cases)
    E = sum(c.mesh.ne for c in cases)
    M = cases[0].params.M
    desc = {"workload": f"batched ensemble of {len(cases)} closed basins (jittered Delaunay, log-uniform "
                        f"2e4-4e5 vertices x {scale:g}, seeded depths 1000-5000 m, eta bumps 0.5 m), M={M}, "
                        f"per-basin dt from the stability rule, one upload and one advance per step",
            "V": V, "E": E, "M": M, "nbasin": len(cases)}
    return cases, desc


def ensemble_oracle_sample(cases, substeps, budget_s=None, rounds=None, oms=None):
    """The FP64 oracle on the ensemble: `substeps` substeps (dt = tau/M of each basin) of every basin
    in turn, for budget_s seconds or `rounds` passes over the basins. Returns (vertex-substeps, s)."""
    from oracle import runner as orc
    from paper_2311_08241_gb300 import inputs as I

    oms = oms or [orc.OracleMesh(c.mesh) for c in cases]
    state = [(c.eta0.copy(), c.U0.copy()) for c in cases]
    work, t0, n = 0, time.perf_counter(), 0
    while True:
        for b, (c, om) in enumerate(zip(cases, oms)):
            p = c.params
            sp = I.Params(g=p.g, theta=p.theta, tau=p.tau / p.M * substeps, M=substeps, nonlinear_h=p.nonlinear_h)
            eta, U, _, _ = om.advance(c.R, sp, 1, *state[b])
            state[b] = (eta, U)
            work += c.mesh.nv * substeps
            if budget_s is not None and time.perf_counter() - t0 >= budget_s:
                return work, time.perf_counter() - t0
        n += 1
        if rounds is not None and n >= rounds:
            return work, time.perf_counter() - t0


def cpu_baseline_ensemble(cases, seconds):
    """The FP64 oracle, as it stands, on the host cores, on a bounded sample of the batched workload:
    4 substeps of each basin in turn until `seconds` elapse (all cores), then a shorter single-thread
    sample."""
    from oracle import runner as orc

    oms = [orc.OracleMesh(c.mesh) for c in cases]
    cores = orc.set_threads(0)
    work, dt = ensemble_oracle_sample(cases, 4, budget_s=seconds, oms=oms)
    orc.set_threads(1)
    work1, dt1 = ensemble_oracle_sample(cases, 4, budget_s=max(1.0, seconds / 4), oms=oms)
    orc.set_threads(cores)
    for om in oms:
        om.close()
    return {"value": work / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "single_thread_value": work1 / dt1, "cpu_model": cpu_model(),
            "sample": f"{work:.4g} vertex-substeps: 4 substeps of each basin of the batch in turn for {dt:.1f} s "
                      f"wall, FP64, OpenMP over {cores} threads; single thread: {work1:.4g} in {dt1:.1f} s"}


def e2e_pipeline(sim, R_h, outs, nsteps):
    """nsteps steps through the public API with host buffers: each uploads its forcing, advances and
    reads back eta and <<U>>; the asynchronous calls pipeline the transfers on the library's copy
    streams, outputs double-buffered (each waited for two steps later)."""
    tickets = [0, 0]
    for n in range(nsteps):
        k = n & 1
        if n >= 2:
            sim.sesw_wait(tickets[k])
        sim.sesw_set_forcing_async(R_h)
        sim.sesw_advance(1)
        tickets[k] = sim.sesw_get_state_async(outs[k][0], None, outs[k][1])
    sim.sesw_wait(0)


def run_ensemble(args, world, rank, local):
    """Batched ensemble: every basin in one upload and one advance per step (layout picked by the
    autotuner), timed on the device; the same through the public API with host buffers; against
    advancing each basin in its own context one after another (bitwise the same results)."""
    import torch

    from paper_2311_08241_gb300 import autotune as AT
    from paper_2311_08241_gb300 import sesw as S

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    cases, desc = ensemble_workload(rank, args.ensemble_basins, args.ensemble_scale)
    meshes = [c.mesh for c in cases]
    params = [c.params for c in cases]
    V, E, M = desc["V"], desc["E"], desc["M"]
    R = np.concatenate([c.R for c in cases])
    eta0 = np.concatenate([c.eta0 for c in cases])
    U0 = np.concatenate([c.U0 for c in cases])
    if args.autotune == "none":
        forms = {"same": -1, "auto": S.SESW_FORM_AUTO, "registers": S.SESW_FORM_REGISTERS,
                 "stream": S.SESW_FORM_STREAM, "stream-uncached": S.SESW_FORM_STREAM_UNCACHED}
        best, table = AT.Choice(S.SESW_MODE_PERSISTENT, blocks_per_sm=args.blocks_per_sm or 1,
                                large_bps=args.large_bps, large_form=forms[args.large_form]), []
    elif args.autotune == "quick":
        best, table = AT.autotune(meshes, params, forcing=R, steps=3, warmup=1, device=local,
                                  graph_patches=(1024,), graph_threads=(512,), wave_sizes=False)
    else:
        best, table = AT.autotune(meshes, params, forcing=R, steps=3, warmup=1, device=local)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(advance, nsteps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            advance()
            b.record(stream)
        torch.cuda.synchronize(dev)
        return [a.elapsed_time(b) for a, b in ev]

    sim = S.Subcycle(local, stream=stream)
    best.apply(sim)
    sim.sesw_mesh_upload_batch(meshes)
    sim.sesw_set_params_batch(params)
    sim.sesw_set_forcing(R)
    sim.sesw_set_state(eta0, U0)
    info = sim.sesw_get_info()
    for _ in range(args.warmup):
        flush.zero_()
        sim.sesw_advance(1)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    step_ms = timed(lambda: sim.sesw_advance(1), args.steps)
    barrier(world)
    clk = clocks.stop()
    if sim.sesw_status() != S.SESW_OK:
        raise RuntimeError("batched run flagged a device status")
    total_ms = reduce_max(sum(step_ms), world, dev)
    value = whole_job_value(V, M, args.steps, world, total_ms)

    # End to end through the public API with pinned host buffers: each step uploads its forcing
    # (every basin), advances the batch, and reads back eta and <<U>> of every basin; the
    # asynchronous calls pipeline the transfers on the library's copy streams.
    R_h = torch.from_numpy(np.ascontiguousarray(R)).pin_memory()
    outs = [(torch.empty(V, dtype=torch.float64).pin_memory(), torch.empty((E, 2), dtype=torch.float64).pin_memory())
            for _ in range(2)]
    n_e2e = max(1, min(args.e2e_steps, args.steps))
    e2e_pipeline(sim, R_h, outs, 2)    # untimed: the copy streams and staging buffers are set up
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e2e_pipeline(sim, R_h, outs, n_e2e)
    e2e_s = reduce_max(time.perf_counter() - t0, world, dev)
    e2e = {"value": world * V * M * n_e2e / e2e_s, "unit": METRIC, "h2d_bytes_per_step": int(R_h.numel() * 8),
           "d2h_bytes_per_step": int(outs[0][0].numel() * 8 + outs[0][1].numel() * 8), "steps": n_e2e,
           "calls": "sesw_set_forcing_async, sesw_advance, sesw_get_state_async on the whole batch "
                    "(pipelined, pinned host buffers)"}

    # the same basins advanced one context after another (each as the library runs a single mesh)
    compare = args.sequential_steps > 0
    singles = []
    for c in cases if compare else []:
        s1 = S.Subcycle(local, stream=stream)
        s1.sesw_mesh_upload(c.mesh)
        s1.sesw_set_params(c.params)
        s1.sesw_set_forcing(c.R)
        s1.sesw_set_state(c.eta0, c.U0)
        singles.append(s1)
    batched_vs_sequential = None
    if compare:
        for s1 in singles:
            s1.sesw_advance(1)
        nseq = max(1, min(args.sequential_steps, args.steps))
        seq_ms = timed(lambda: [s1.sesw_advance(1) for s1 in singles], nseq)
        speedup = statistics.mean(seq_ms) / statistics.mean(step_ms)
        # SSH of the two forms after the same steps from the same start: bitwise equal
        nchk = 5
        sim.sesw_set_state(eta0, U0)
        sim.sesw_advance(nchk)
        eta_b = sim.sesw_get_state()[0]
        eta_s = []
        for c, s1 in zip(cases, singles):
            s1.sesw_set_state(c.eta0, c.U0)
            s1.sesw_advance(nchk)
            eta_s.append(s1.sesw_get_state()[0])
            s1.close()
        eta_s = np.concatenate(eta_s)
        batched_vs_sequential = {"speedup": speedup, "sequential_ms_per_step": statistics.mean(seq_ms),
                                 "batched_ms_per_step": statistics.mean(step_ms),
                                 "max_ssh_difference_m": float(np.max(np.abs(eta_b - eta_s))),
                                 "bitwise_equal": bool(np.array_equal(eta_b, eta_s)), "after_steps": nchk}

    persistent = info["mode"] == S.SESW_MODE_PERSISTENT
    mean_step_s = statistics.mean(step_ms) * 1e-3
    b_alg_step = algorithmic_bytes_per_substep(V, E) * M
    launches_per_step = max(1, sim.sesw_get_info()["launches"])
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if persistent:
        kernels = ("k_persistent", "k_persistent_stream")
        fig = profile_figures("k_persistent_ensemble", kernels, layout=best.label())
        roofline = roofline_issue(f"k_persistent + k_persistent_stream ({info['npack']} packs in "
                                  f"{launches_per_step} launches per step)",
                                  mean_step_s, fig and fig.get("warp_instructions_per_step"),
                                  fig and fig.get("dram_bytes_per_step"), b_alg_step, sms, sm_max_mhz_of(clk),
                                  per="step")
        if fig:
            roofline["profile"] = fig["profile"]
    else:
        achieved = b_alg_step / mean_step_s / 1e9
        peak, src = measured_hbm_peak()
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": None, "peak_source": src, "kernel": "k_substep", "bytes_per_step": b_alg_step}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(desc, layout=best.label(), npatch=info["npatch"], nslot=info["nslot"],
                           npack=info["npack"], streamed_first_pack=info["streamed"],
                           l2="flushed between timed steps (256 MiB write)", parallelism=f"replicas{world}",
                           autotune=args.autotune,
                           autotune_ms_per_step={c.label(): t for c, t in table}),
            "roofline": roofline, "e2e": e2e,
            "batched_vs_sequential": batched_vs_sequential,
            "gpu_launches": args.steps * launches_per_step,
            "graph_launches_per_step": 1 if sim.sesw_get_info()["step_graph"] else 0,
            "clocks": clk}
    sim.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_ensemble(cases, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_surrogate(args, world, rank, local):
    """Learned surrogate on the global-like sphere: data from the plain subcycle, training on the GPU,
    held-out loss against persistence, rollouts against the plain subcycle (and fewer substeps)."""
    import torch

    from paper_2311_08241_gb300 import inputs as I
    from paper_2311_08241_gb300 import sesw as S
    from paper_2311_08241_gb300 import surrogate as SG

    torch.cuda.set_device(local)
    case = I.sphere_case(level=args.surrogate_level, nsteps=args.surrogate_steps)
    V, E, M = case.mesh.nv, case.mesh.ne, case.params.M
    ntraj, nst = args.surrogate_traj, args.surrogate_steps
    base_seed = 20231119 + 1000 * rank
    forcing = lambda k: SG.sphere_forcing(case, base_seed + k)
    sim = S.Subcycle(local)
    sim.sesw_mesh_upload(case.mesh)
    sim.sesw_set_params(case.params)
    sim.sesw_surrogate_init(ntraj * nst, seed=1)
    t0 = time.perf_counter()
    SG.generate(sim, case.mesh, forcing, ntraj, nst)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    sp = SG.split(ntraj, nst)
    xy = case.mesh.xy
    edge = float(np.sqrt(np.mean((xy[:, 1] - xy[:, 0]) ** 2 * 2)))
    sim.sesw_surrogate_fit_scales(ntraj * nst, edge)
    baseline = SG.persistence_loss(sim, sp.test)
    untrained = sim.sesw_surrogate_loss(sp.test)
    t0 = time.perf_counter()
    hist = SG.train(sim, sp.train, args.surrogate_epochs, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    test_loss = sim.sesw_surrogate_loss(sp.test)
    weights = sim.sesw_surrogate_weights()
    scales = sim.sesw_surrogate_scales()
    sim.close()
    k_test = ntraj - 1
    roll = SG.rollout_error(case, forcing(k_test), case.params, weights, scales, nst, args.resid_tol,
                            coarse_M=(M // 2,), device=local)
    plain_ms = roll["plain"]["ms_per_step"]
    sur_ms = roll["surrogate"]["ms_per_step"]
    line = {"metric": METRIC, "value": V * M / (sur_ms * 1e-3), "unit": METRIC, "n_gpus": 1,
            "steps": nst, "warmup": 1, "ms_per_step": sur_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 weights, f32 accumulate", "data": "synthetic",
            "config": {"workload": f"learned surrogate on the icosahedral sphere level {args.surrogate_level} "
                                   f"(V={V}, E={E}, M={M}, tau={case.params.tau:g} s)",
                       "samples": ntraj * nst, "trajectories": ntraj, "held_out_trajectories": int(sp.ntraj - len(sp.train) // nst),
                       "epochs": args.surrogate_epochs, "resid_tol": args.resid_tol},
            "surrogate": {"held_out_loss": test_loss, "persistence_loss": baseline, "untrained_loss": untrained,
                          "loss_ratio_vs_persistence": test_loss / baseline, "train_loss_per_epoch": hist,
                          "generate_s": t_gen, "train_s": t_train,
                          "speedup_vs_plain": plain_ms / sur_ms, "rollout": roll,
                          "gain_over_plain": SG.gain_summary(roll),
                          "ssh_signal_m": roll["max_ssh_reference_m"]},
            "gpu_launches": roll["surrogate"]["gpu_launches"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args, world, rank):
    """The oracle on the host cores, on bounded samples of the same workload."""
    if rank != 0:
        return
    from oracle import runner as orc
    from paper_2311_08241_gb300 import inputs as I

    if args.workload == "ensemble":
        cases, desc = ensemble_workload(0, args.ensemble_basins, args.ensemble_scale)
        S = max(1, args.ref_substeps)
        oms = [orc.OracleMesh(c.mesh) for c in cases]
        cores = orc.set_threads(0)
        ensemble_oracle_sample(cases, S, rounds=args.warmup, oms=oms) if args.warmup else None
        work, dt = ensemble_oracle_sample(cases, S, rounds=args.steps, oms=oms)
        value = work / dt
        sample_txt = (f"each step: {S} substeps (dt = tau/M of each basin) of every basin of the batch, FP64 "
                      f"oracle, OpenMP over {cores} threads")
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": dict(desc, sample_substeps_per_step=S),
                "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                                 "sample": sample_txt},
                "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "gpu_launches": 0}
        print(json.dumps(line), flush=True)
        return
    case, desc = workload(args.workload)
    S = max(1, args.ref_substeps)
    p = case.params
    sample = I.Params(g=p.g, theta=p.theta, tau=p.tau / p.M * S, M=S, nonlinear_h=p.nonlinear_h)
    om = orc.OracleMesh(case.mesh)
    cores = orc.set_threads(0)
    eta, U = case.eta0.copy(), case.U0.copy()
    for _ in range(args.warmup):
        eta, U, _, _ = om.advance(case.R, sample, 1, eta, U)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        eta, U, _, _ = om.advance(case.R, sample, 1, eta, U)
    dt = time.perf_counter() - t0
    value = case.mesh.nv * S * args.steps / dt
    sample_txt = (f"each step: {S} substeps (dt = tau/M = {p.tau / p.M:g} s) of the benchmark mesh, FP64 "
                  f"oracle, OpenMP over {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(desc, sample_substeps_per_step=S),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample_txt},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch

    from paper_2311_08241_gb300 import sesw as S

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case, desc = workload(args.workload)
    if args.scheme == "sesm":
        from paper_2311_08241_gb300 import inputs as I

        p = case.params
        case.params = I.Params(g=p.g, theta=p.theta, tau=p.tau, M=p.M, nonlinear_h=p.nonlinear_h, scheme=1)
        desc = dict(desc, scheme="SESM (AB3-AM4, Eqs. 4.7-4.8)")
    W = None
    if args.freshwater:
        W = args.freshwater * (0.3 + np.random.default_rng(20231119).standard_normal(case.mesh.nv))
        desc = dict(desc, freshwater=f"W = {args.freshwater:g} m/s x (0.3 + N(0,1)), seeded (Eq. 4.5)")
    if args.visc:
        from paper_2311_08241_gb300 import inputs as I

        p = case.params
        if args.visc == "auto":
            stiff = S.sesw_mesh_check(case.mesh)["visc_stiffness"]
            visc = (0.2 / (p.tau / p.M * stiff), 1.0)
        else:
            visc = tuple(float(x) for x in args.visc.split(","))
        case.params = I.Params(g=p.g, theta=p.theta, tau=p.tau, M=p.M, nonlinear_h=p.nonlinear_h,
                               scheme=p.scheme, visc=visc)
        args.mode = "graph"
        desc = dict(desc, viscosity=f"A = {visc[0]:.4g} m^2/s + {visc[1]:g} |du| L (Eq. viscosity_BT)")
    V, E, M = case.mesh.nv, case.mesh.ne, case.params.M
    stream = torch.cuda.current_stream(dev)
    sim = S.Subcycle(local, stream=stream)
    sim.sesw_set_mode({"auto": S.SESW_MODE_AUTO, "graph": S.SESW_MODE_GRAPH,
                       "persistent": S.SESW_MODE_PERSISTENT}[args.mode])
    sim.sesw_set_persistent_form({"auto": S.SESW_FORM_AUTO, "registers": S.SESW_FORM_REGISTERS,
                                  "stream": S.SESW_FORM_STREAM,
                                  "stream-uncached": S.SESW_FORM_STREAM_UNCACHED}[args.persistent_form])
    pv = args.patch_vertices
    if pv is None:
        if args.visc:
            # the fused viscosity substep (56 registers x 256 threads) keeps 4 blocks per SM:
            # patches sized so that the channel is exactly one wave of them
            from paper_2311_08241_gb300.autotune import wave_patch_sizes

            nsm = torch.cuda.get_device_properties(dev).multi_processor_count
            pv = wave_patch_sizes(V, nsm, (4,))[0]
        else:
            pv = 256
    sim.sesw_set_patch_vertices(pv)
    sim.sesw_set_block_threads(args.block_threads)
    sim.sesw_set_blocks_per_sm(args.blocks_per_sm)
    sim.sesw_mesh_upload(case.mesh)
    sim.sesw_set_params(case.params)
    sim.sesw_set_forcing(case.R)
    if W is not None:
        sim.sesw_set_freshwater(W)
    sim.sesw_set_state(case.eta0, case.U0)
    info = sim.sesw_get_info()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        flush.zero_()
        sim.sesw_advance(1)
    torch.cuda.synchronize(dev)
    if sim.sesw_status() != S.SESW_OK:
        raise RuntimeError("warm-up went unstable")

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    for k in range(args.steps):
        flush.zero_()                       # L2 flushed between timed steps
        ev[k][0].record(stream)
        sim.sesw_advance(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    rc = sim.sesw_status()
    if rc != S.SESW_OK:
        raise RuntimeError(f"timed run flagged status {rc}")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = reduce_max(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_value(V, M, args.steps, world, total_ms)

    # Roofline of the dominant kernel. Persistent mode: one k_persistent launch per step
    # does all M substeps, so a launch moves M * B_alg algorithmic bytes. Graph mode: M
    # k_substep launches per step, each B_alg (the step's short epilogue launch is
    # included in the event time, which understates the kernel's rate).
    # SESM: the same with its own byte count per substep (persistent: one k_persistent_sesm
    # launch per step; graph: M + 1 k_sesm launches). Viscosity (graph): fused into the
    # substep kernel, rated per substep with the bytes it adds.
    persistent = info["mode"] == S.SESW_MODE_PERSISTENT
    if args.scheme == "sesm":
        b_alg = sesm_bytes_per_substep(V, E)
    else:
        b_alg = algorithmic_bytes_per_substep(V, E)
    if args.visc:
        b_alg += viscosity_bytes_per_substep(V, E)
    mean_step_s = statistics.mean(step_ms) * 1e-3
    per_launch = b_alg * M if persistent else b_alg
    launch_s = mean_step_s if persistent else mean_step_s / M
    achieved = per_launch / launch_s / 1e9
    peak, peak_src = measured_hbm_peak()
    if args.scheme == "sesm":
        kname = ("k_persistent_sesm_stream" if info["streamed"] else "k_persistent_sesm") if persistent else "k_sesm"
    else:
        kname = ("k_persistent_stream" if info["streamed"] else "k_persistent") if persistent else "k_substep"
    if args.visc:
        kname = "k_substep (viscosity fused)"
    if persistent:
        # on chip for the M substeps of a launch: bound by instruction issue, not by DRAM
        fig = profile_figures(f"{kname}_{args.workload}", (kname,))
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        model = "24 V + 108 E per substep" if args.scheme == "sesm" else "12 V + 92 E per substep"
        roofline = roofline_issue(kname, launch_s, fig and fig.get("warp_instructions_per_launch"),
                                  fig and fig.get("dram_bytes_per_launch"), per_launch, sms, sm_max_mhz_of(clk),
                                  alg_model=model)
        if fig:
            roofline["profile"] = fig["profile"]
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": profiled_traffic_for(kname, args.workload), "peak_source": peak_src,
                    "kernel": kname, "bytes_per_launch": per_launch}

    # End to end through the public API with pinned host buffers: each step uploads its
    # forcing, advances, and reads back eta and <<U>>. The asynchronous calls pipeline the
    # transfers on the library's copy streams (outputs double-buffered, each waited for two
    # steps later); the synchronous calls are timed too.
    R_h = torch.from_numpy(np.ascontiguousarray(case.R)).pin_memory()
    outs = [(torch.empty(V, dtype=torch.float64).pin_memory(), torch.empty((E, 2), dtype=torch.float64).pin_memory())
            for _ in range(2)]
    n_e2e = max(1, min(args.e2e_steps, args.steps))
    e2e_pipeline(sim, R_h, outs, 2)    # untimed: the copy streams and staging buffers are set up
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e2e_pipeline(sim, R_h, outs, n_e2e)
    e2e_s = reduce_max(time.perf_counter() - t0, world, dev)
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        sim.sesw_set_forcing(R_h)
        sim.sesw_advance(1)
        sim.sesw_get_state(outs[0][0], None, outs[0][1])
    sync_s = reduce_max(time.perf_counter() - t0, world, dev)
    e2e = {"value": world * V * M * n_e2e / e2e_s, "unit": METRIC, "h2d_bytes_per_step": int(R_h.numel() * 8),
           "d2h_bytes_per_step": int(outs[0][0].numel() * 8 + outs[0][1].numel() * 8), "steps": n_e2e,
           "calls": "sesw_set_forcing_async, sesw_advance, sesw_get_state_async (pipelined, pinned host buffers)",
           "synchronous_value": world * V * M * n_e2e / sync_s}

    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(desc, mode="persistent" if persistent else "graph",
                           patch_vertices=info["patch_vertices"], block_threads=info["block_threads"],
                           blocks_per_sm=info["blocks_per_sm"], slots_per_thread=info["slots_per_thread"],
                           smem_cached=info["cached"],
                           npatch=info["npatch"],
                           nslot=info["nslot"], l2="flushed between timed steps (256 MiB write)",
                           parallelism=f"replicas{world}"),
            "roofline": roofline, "e2e": e2e,
            "gpu_launches": args.steps * (1 if persistent else (M + 1 if args.scheme == "sesm" else M) + 1),
            "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(case, args.cpu_seconds, rank, W=W)
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.gpus != world and world > 1:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE {world}", file=sys.stderr)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        elif args.workload == "ensemble":
            run_ensemble(args, world, rank, local)
        elif args.workload == "surrogate":
            run_surrogate(args, world, rank, local)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
