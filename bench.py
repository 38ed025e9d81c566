#!/usr/bin/env python
"""Benchmark of the long-range planewave-DF Coulomb build (steps a2..a8).

Workload: diamond-like cubic cell a = 6.74 bohr, 8 carbon-like centres,
spherical s8 p4 d2 per centre (240 AOs), k-mesh 4x4x4 (64 Hermitian,
time-reversal-symmetric D^k from 16 random occupied orbitals), omega = 0.4,
exp(-G^2/4w^2) > 1e-14, primitive pairs kept above overlap 1e-12.

One step = one whole build from D^k (resident in HBM) to J^k and E_J.
Metric value = pair*G evaluations per second, the unit being one ordered
screened primitive-shell pair times one G != 0 of the full sphere.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica of the workload (the bench
workload is one cell); value is the whole-job rate, timed as the max over
ranks.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LR J-build ms & pair·G evals/s, split-prec vs FP64 form at max|ΔJ|≤1e-8 Eh"
UNIT = "pair*G/s"
WORKLOAD = ("diamond-like cubic a=6.74 bohr, 8 C-like centres, spherical s8p4d2 (240 AOs), "
            "k 4x4x4 (64 D^k, 16 occupied), omega 0.4, exp(-G^2/4w^2)>1e-14, pair overlap>1e-12")
L2_FLUSH_BYTES = 512 << 20
PAIR_GCUT_EPS = 1e-12  # the per-pair G cutoff variant (screening threshold of Sec. 2.5)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batch, molecular-crystal and slab legs")
    ap.add_argument("--leg", choices=["batch", "molecular_crystal", "slab"], default=None,
                    help="run only this extra workload (one GPU, rank 0) and print its JSON; for profiling")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                rows.append(parts)
            except ValueError:
                pass
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (the time of the slowest replica); x itself
    without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_replica, seconds):
    """Units of all replicas per second of the slowest one."""
    return world * units_per_replica / seconds


def walk_flops(info, ndens, form):
    """Algorithmic flops of one walk launch (structure-factor or back-contraction
    pass; both have the same count).  Per (pair record of class L, half-sphere G):
    FP64 form: 4L + 14 flops (an (L+1)-term complex Horner, prefactor x phase
    and the accumulation); split form: the same arithmetic evaluated in
    double-float on the FP32 pipe (an FMA counts two): L Horner or accumulation
    steps of 38, one complex double-float product of 50 (prefactor x
    polynomial) and one complex double-float sum of 22; where the n1 recurrence
    runs (no per-record X(n1) table) each point also advances the prefactor and
    its ratio, another complex product of 50 and a complex-by-real one of 20.
    So 38L + 72 with the table, 38L + 142 without."""
    if form == "fp64":
        per = lambda L: 4 * L + 14
    elif info.get("n1_table", 0) > 0:
        per = lambda L: 38 * L + 72
    else:
        per = lambda L: 38 * L + 142
    return ndens * sum(n * info["ng_half"] * per(L) for L, n in enumerate(info["pairs_by_class"]))


def traffic_from_profile(kernel: str):
    """dram bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (its recorded source hash must match)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_diamond240_k444.md")
    src_name = "walk_split.cu" if kernel.endswith("_split") else "walk.cu"
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{16,64})", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m or not t:
        return None
    src = open(os.path.join(ROOT, "paper_2509_16460_gb300", "csrc", src_name), "rb").read()
    if hashlib.sha256(src).hexdigest()[:len(m.group(1))] != m.group(1):
        return None
    return float(t.group(1))


def cpu_oracle_run(w, pair_stride):
    import oracle
    r = oracle.lrj(w, pair_stride=pair_stride, want_j0n=False, want_rho=False)
    threads = os.cpu_count() or 1
    try:
        import ctypes
        gomp = ctypes.CDLL("libgomp.so.1")
        threads = int(gomp.omp_get_max_threads())
    except OSError:
        pass
    units = r["units"] * w.ndens
    return r, units, threads


def time_events(fn, steps, flush, stream):
    """Mean device ms of fn() over `steps` calls, L2 flushed before each."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def batch_leg(ftcj, W, torch, flush, steps):
    """The uneven batch: 64 independent triclinic cells, walk shapes picked by
    the autotuner, the whole batch captured once into a CUDA graph and
    replayed; beside it the same cells built one after another on one stream."""
    import numpy as np
    cells = W.cfg4()
    Dks = [torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda() for w in cells]
    out = {"workload": "64 seeded triclinic cells, edges 6-16 bohr, 2-24 centres (H/C/O/Mg-like templates), "
                       "k-meshes 1..3 per axis, omega 0.3-0.5",
           "ncell": len(cells)}
    t0 = time.perf_counter()
    B = ftcj.Batch(cells, precision=ftcj.FTCJ_PREC_SPLIT, autotune=True)
    out["setup_s_with_autotune"] = time.perf_counter() - t0
    units = sum(float(i["pair_g_units"]) * w.ndens for i, w in zip(B.infos, cells))
    out["pair_g_units_per_step"] = units
    s = torch.cuda.Stream()
    Jg, Eg = B.outputs_like(Dks)
    torch.cuda.synchronize()
    B.capture(Dks, Jg, Eg, stream=s)
    for _ in range(3):
        B.replay(stream=s)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        ms = time_events(lambda: B.replay(stream=s), steps, flush, s)
    out["graph_replay"] = {"ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT}
    stream = torch.cuda.current_stream()
    plans = [ftcj.Plan.from_workload(w, precision=ftcj.FTCJ_PREC_SPLIT) for w in cells]
    outs = [p.jbuild(D) for p, D in zip(plans, Dks)]

    def serial():
        for p, D, (J, E) in zip(plans, Dks, outs):
            p.jbuild(D, J, E)
    for _ in range(3):
        serial()
    ms_serial = time_events(serial, steps, flush, stream)
    out["serial_one_stream"] = {"ms_per_step": ms_serial, "value": units / (ms_serial * 1e-3), "unit": UNIT}
    out["max_abs_dJ_graph_vs_serial"] = max(float((a - b[0]).abs().max()) for a, b in zip(Jg, outs))
    for p in plans:
        p.close()
    B.close()
    return out


def cfg3_leg(ftcj, W, torch, flush, steps):
    """The molecular-crystal cell (1056 AOs, k 2x2x2, 2 spin densities in one
    call), split and FP64 forms, and the split form with the autotuned walk shape."""
    import numpy as np
    w = W.cfg3()
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    out = {"workload": "orthorhombic 14.0x17.8x12.9 bohr, 4 six-rings (24 C-like, 24 H-like), 1056 spherical AOs, "
                       "k 2x2x2, 2 spin densities x 8 D^k, omega 0.5", "ndens": w.ndens}
    stream = torch.cuda.current_stream()
    res = {}
    for form, prec, eps in (("split", ftcj.FTCJ_PREC_SPLIT, 0.0), ("fp64", ftcj.FTCJ_PREC_FP64, 0.0),
                            ("split_pair_gcut", ftcj.FTCJ_PREC_SPLIT, PAIR_GCUT_EPS)):
        p = ftcj.Plan.from_workload(w, precision=prec, pair_gcut_eps=eps)
        units = float(p.info["pair_g_units"]) * w.ndens
        J, E = p.jbuild(Dk)
        for _ in range(2):
            p.jbuild(Dk, J, E)
        ms = time_events(lambda: p.jbuild(Dk, J, E), steps, flush, stream)
        out[form] = {"ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT}
        if eps > 0:
            out[form]["pair_gcut_eps"] = eps
            out[form]["walked_fraction_of_units"] = p.info["pair_g_units_walked"] / p.info["pair_g_units"]
        out["pair_g_units_per_step"] = units
        res[form] = (J.clone(), E.clone())
        p.close()
    # the same split build with the walk shape picked by the autotuner
    t0 = time.perf_counter()
    chunk, rb, _ = ftcj.autotune(w, precision=ftcj.FTCJ_PREC_SPLIT)
    tune_s = time.perf_counter() - t0
    p = ftcj.Plan.from_workload(w, precision=ftcj.FTCJ_PREC_SPLIT, chunk_points=chunk, rho_blocks=rb)
    J, E = p.jbuild(Dk)
    for _ in range(2):
        p.jbuild(Dk, J, E)
    ms = time_events(lambda: p.jbuild(Dk, J, E), steps, flush, stream)
    out["split_autotuned"] = {"ms_per_step": ms, "value": out["pair_g_units_per_step"] / (ms * 1e-3), "unit": UNIT,
                              "chunk_points": chunk, "rho_blocks": rb, "shape_note": "0 = the plan's own default",
                              "autotune_s": tune_s,
                              "max_abs_dJ_vs_split_default": float((J - res["split"][0]).abs().max())}
    p.close()
    out["split_pair_gcut_vs_fp64_max_abs_dJ"] = float((res["split_pair_gcut"][0] - res["fp64"][0]).abs().max())
    out["split_vs_fp64_max_abs_dJ"] = float((res["split"][0] - res["fp64"][0]).abs().max())
    out["split_vs_fp64_abs_dEJ"] = float((res["split"][1] - res["fp64"][1]).abs().max())
    out["split_speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["split"]["ms_per_step"]
    return out


def slab_leg(ftcj, W, torch, flush, steps):
    """The surface slab (rock-salt 2x2 (001), 4 layers + CO, 1270 AOs, k
    3x3x1): split and FP64 builds, and the split plan's nuclear gradient
    (dE_J/dR of every centre)."""
    import numpy as np
    w = W.cfg5()
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    out = {"workload": "rock-salt (001) 2x2 slab, 4 layers (16 Mg-like + 16 O-like) + CO, 20 bohr vacuum, "
                       f"{w.nao} spherical AOs, k 3x3x1, omega 0.4", "ndens": w.ndens}
    stream = torch.cuda.current_stream()
    res = {}
    for form, prec in (("split", ftcj.FTCJ_PREC_SPLIT), ("fp64", ftcj.FTCJ_PREC_FP64)):
        p = ftcj.Plan.from_workload(w, precision=prec)
        units = float(p.info["pair_g_units"]) * w.ndens
        out["pair_g_units_per_step"] = units
        J, E = p.jbuild(Dk)
        for _ in range(2):
            p.jbuild(Dk, J, E)
        ms = time_events(lambda: p.jbuild(Dk, J, E), steps, flush, stream)
        out[form] = {"ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT}
        res[form] = (J.clone(), E.clone())
        if form == "split":
            EJ, G = p.grad(Dk)
            for _ in range(2):
                p.grad(Dk, EJ, G)
            ms = time_events(lambda: p.grad(Dk, EJ, G), steps, flush, stream)
            torch.cuda.synchronize()
            out["gradient"] = {"ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT,
                               "note": "one call: fold, Hermite map and rho pass of the plan's form, the adjoint "
                                       "walk of degree L+1 (double-float where grad_split is 1), then the FP64 "
                                       "per-centre assembly",
                               "grad_split": int(p.info["grad_split"]),
                               "abs_dEJ_vs_build": float((EJ - E).abs().max()),
                               "max_abs_force": float(G.abs().max()),
                               "sum_of_forces_max_abs": float(G.sum(dim=1).abs().max())}
        p.close()
    out["split_vs_fp64_max_abs_dJ"] = float((res["split"][0] - res["fp64"][0]).abs().max())
    out["split_vs_fp64_abs_dEJ"] = float((res["split"][1] - res["fp64"][1]).abs().max())
    out["split_speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["split"]["ms_per_step"]
    return out


def run_reference(args, world, rank):
    """The reference arm is the CPU oracle, timed as it stands on the host cores."""
    if rank != 0:
        return 0
    import oracle
    from paper_2509_16460_gb300 import workloads as W
    oracle.build()
    w = W.cfg2()
    stride = 8
    for _ in range(args.warmup):
        cpu_oracle_run(w, stride)
    times, units = [], 0.0
    threads = 1
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r, units, threads = cpu_oracle_run(w, stride)
        times.append(time.perf_counter() - t0)
    mean = statistics.mean(times)
    value = units / mean
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "fp64 CPU oracle",
                   "sample": f"every {stride}th ordered primitive pair, all G (stride {stride})"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"every {stride}th ordered screened primitive pair of the workload, full G sphere"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_16460_gb300 import ftcj
    from paper_2509_16460_gb300 import workloads as W

    torch.cuda.set_device(local)
    if args.leg:
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        legs = {"batch": batch_leg, "molecular_crystal": cfg3_leg, "slab": slab_leg}
        print(json.dumps({"leg": args.leg, **legs[args.leg](ftcj, W, torch, flush, args.steps)}), flush=True)
        return 0
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = W.cfg2()
    stream = torch.cuda.current_stream()
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    peaks = {"fp64": ftcj.probe_fma_peak(0), "split": ftcj.probe_fma_peak(1)}
    forms = {}
    infos = {}
    results = {}
    for form, prec, eps in (("split", ftcj.FTCJ_PREC_SPLIT, 0.0), ("fp64", ftcj.FTCJ_PREC_FP64, 0.0),
                            ("split_pair_gcut", ftcj.FTCJ_PREC_SPLIT, PAIR_GCUT_EPS)):
        plan = ftcj.Plan.from_workload(w, precision=prec, pair_gcut_eps=eps)
        info = plan.info
        units = float(info["pair_g_units"]) * w.ndens
        Jk = torch.empty_like(Dk)
        EJ = torch.empty(w.ndens, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            plan.jbuild(Dk, Jk, EJ)
        torch.cuda.synchronize()
        # timed region: device time per step, L2 flushed between steps
        plan.profile_enable(args.steps)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        sampler = ClockSampler(local)
        barrier()
        sampler.start()
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            plan.jbuild(Dk, Jk, EJ)
            ev[k][1].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall0
        clocks = sampler.stop()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        phase_ms, batches, launches = plan.profile_read()
        plan.profile_enable(0)
        ms = max_over_ranks(statistics.mean(step_ms), dist, "cuda")
        value = whole_job_rate(world, units, ms * 1e-3)
        # end to end through the host-buffer entry point
        Dk_h = torch.from_numpy(np.ascontiguousarray(w.Dk)).pin_memory()
        Jk_h = torch.empty(Dk_h.shape, dtype=torch.complex128).pin_memory()
        EJ_h = torch.empty(w.ndens, dtype=torch.float64).pin_memory()
        plan.jbuild_host(Dk_h, Jk_h, EJ_h)
        e2e_t = []
        barrier()
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.jbuild_host(Dk_h, Jk_h, EJ_h)
            e2e_t.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(statistics.mean(e2e_t), dist, "cuda")
        # roofline of the dominant kernel: FP64 pipe (fp64) or FP32 pipe (split)
        pipe_form = "fp64" if form == "fp64" else "split"
        suffix = "_split" if pipe_form == "split" else ""
        walks = {"k_rho_walk" + suffix: phase_ms["rho_walk"], "k_j_walk" + suffix: phase_ms["j_walk"]}
        kname = max(walks, key=walks.get)
        per_launch_ms = walks[kname] / max(batches, 1)
        # with per-pair cutoffs the walks evaluate only the walked share of the units
        walked = info["pair_g_units_walked"] / info["pair_g_units"]
        achieved = walk_flops(info, w.ndens, pipe_form) * walked / (per_launch_ms * 1e-3)
        peak = peaks[pipe_form]
        roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic_from_profile(kname) if eps == 0 else None,
                    "kernel": kname, "pipe": "FP64" if pipe_form == "fp64" else "FP32",
                    "peak_source": f"measured {'FP64' if pipe_form == 'fp64' else 'FP32'} FMA throughput "
                                   "(ftcj_probe_fma_peak) on this GPU",
                    "nominal_peak": 152 * 2 * 2.07e9 * (2 if pipe_form == "fp64" else 128) / 1e12,
                    "phase_ms_per_step": {k: v / max(batches, 1) for k, v in phase_ms.items()}}
        if eps > 0:
            roofline["flops_note"] = "algorithmic flops scaled by the walked fraction of the units (per-class mix ignored)"
        forms[form] = {"value": value, "unit": UNIT, "ms_per_step": ms, "step_ms_min": min(step_ms),
                       "e2e": {"value": whole_job_rate(world, units, e2e_s), "unit": UNIT,
                               "ms_per_step": e2e_s * 1e3,
                               "h2d_bytes_per_step": Dk_h.numel() * 16,
                               "d2h_bytes_per_step": Jk_h.numel() * 16 + EJ_h.numel() * 8,
                               "transfer": "pinned host buffers read and written by the device over the host link; "
                                           + ("the split form's fold reads only the upper triangle of the "
                                              "Hermitian D^k" if pipe_form == "split" else
                                              "the whole D^k is read")},
                       "roofline": roofline, "gpu_launches": int(launches), "clocks": clocks,
                       "wall_s_timed_region": t_wall,
                       "walk_shape": {"rho_blocks": info["rho_blocks"], "n1_table": info["n1_table"],
                                      "nchunks": info["nchunks"]}}
        if eps > 0:
            forms[form]["pair_gcut_eps"] = eps
            forms[form]["walked_fraction_of_units"] = walked
            forms[form]["screened_fraction_of_units"] = info["pair_g_units_screened"] / info["pair_g_units"]
        infos[form] = info
        results[form] = (Jk.cpu().numpy(), EJ.cpu().numpy())
        plan.close()

    head = forms["split"]
    info = infos["split"]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2 walks (double-float), f64 setup/sums/E_J", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "split", "pair_g_units_per_step": units,
                   "npairs_ordered": info["npairs_ordered"], "pair_records": info["npairs"],
                   "ng_full": info["ng_full"], "nao": info["nao"], "nk": info["nk"],
                   "records_by_class": info["pairs_by_class"], "rho_blocks": info["rho_blocks"],
                   "n1_table": info["n1_table"],
                   "l2": f"{L2_FLUSH_BYTES >> 20} MB buffer written between timed steps",
                   "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
        "e2e": {k: head["e2e"][k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")},
        "gpu_launches": head["gpu_launches"],
        "roofline": head["roofline"],
        "clocks": head["clocks"],
        "forms": forms,
        "split_speedup_vs_fp64": forms["fp64"]["ms_per_step"] / head["ms_per_step"],
    }

    if rank == 0 and not args.no_extra:
        extra_steps = max(3, min(args.steps, 10))
        line["batch"] = batch_leg(ftcj, W, torch, flush, extra_steps)
        line["workloads"] = {"molecular_crystal": cfg3_leg(ftcj, W, torch, flush, extra_steps),
                             "slab": slab_leg(ftcj, W, torch, flush, extra_steps)}
    if rank == 0 and not args.no_cpu_baseline:
        # the whole oracle on the host cores: the CPU baseline and the accuracy of this run
        r, cu, threads = cpu_oracle_run(w, 1)
        line["cpu_baseline"] = {"value": cu / r["seconds"], "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "the whole workload (every pair, full sphere), one build",
                                "seconds": r["seconds"]}
        for form, (Jg, Eg) in results.items():
            forms[form]["max_abs_dJ_vs_oracle"] = float(np.abs(Jg - r["Jk"]).max())
            forms[form]["abs_dEJ_vs_oracle"] = float(np.abs(Eg - r["EJ"]).max())
        line["max_abs_dJ_vs_oracle"] = forms["split"]["max_abs_dJ_vs_oracle"]
        line["abs_dEJ_vs_oracle"] = forms["split"]["abs_dEJ_vs_oracle"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
