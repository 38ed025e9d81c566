#!/usr/bin/env python
"""Benchmark of the long-range planewave-DF Coulomb build (steps a2..a8).

Headline workload (the largest single-GPU configuration): molecular-crystal
cell, orthorhombic 14.0 x 17.8 x 12.9 bohr, 4 six-rings (24 C-like, 24
H-like centres), 1056 spherical AOs, k-mesh 2x2x2, 2 spin densities x 8 D^k
built in one call, omega 0.5, exp(-G^2/4w^2) > 1e-14, primitive pairs kept
above overlap 1e-12.  The split-precision form is the headline, the FP64 form
is timed beside it; the diamond-like 240-AO cell (k 4x4x4) is a secondary
line, checked whole against the CPU oracle.

One step = one whole build from D^k (resident in HBM) to J^k and E_J.
Metric value = pair*G evaluations per second, the unit being one ordered
screened primitive-shell pair times one G != 0 of the full sphere, times the
densities of the call.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) the build is sharded by pair records over the ranks
(record shards, an all-reduce of rho(G) and one of J^{0n} over NCCL): the
total work is fixed, so scaling is strong, and value is the units of the one
build over the slowest rank's time.
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
WORKLOADS = {
    "molecular_crystal": ("orthorhombic 14.0x17.8x12.9 bohr, 4 six-rings (24 C-like, 24 H-like centres), "
                          "1056 spherical AOs, k 2x2x2, 2 spin densities x 8 D^k in one call, omega 0.5, "
                          "exp(-G^2/4w^2)>1e-14, pair overlap>1e-12"),
    "diamond": ("diamond-like cubic a=6.74 bohr, 8 C-like centres, spherical s8p4d2 (240 AOs), "
                "k 4x4x4 (64 D^k, 16 occupied), omega 0.4, exp(-G^2/4w^2)>1e-14, pair overlap>1e-12"),
}
HEADLINE = "molecular_crystal"
L2_FLUSH_BYTES = 512 << 20
PAIR_GCUT_EPS = 1e-12  # the per-pair G cutoff variant (screening threshold of Sec. 2.5)
CPU_BASELINE_STRIDE = 32   # oracle sample of the ours-arm CPU baseline: every 32nd ordered pair
REFERENCE_STRIDE = 256     # oracle sample per step of the reference arm


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secondary diamond line and the batch and slab legs")
    ap.add_argument("--forms", default="split_tc,split,fp64,split_pair_gcut,fp64_pair_gcut",
                    help="comma list of the headline forms to time (split is always timed)")
    ap.add_argument("--leg", choices=["batch", "molecular_crystal", "slab", "diamond", "gpw"], default=None,
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
            if len(parts) == len(self.FIELDS):
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (the time of the slowest rank); x itself
    without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def strong_rate(units, seconds):
    """Units of the one (sharded) build per second of its slowest rank."""
    return units / seconds


def method_flops_per_unit(L):
    """Algorithmic flops of one (pair record of class L, half-sphere G) per pass
    (structure-factor or back-contraction): an (L+1)-term complex Horner in n1
    (4 flops per term beyond the first), the prefactor x phase product and the
    complex accumulation: 4L + 14, whatever arithmetic the form runs it in."""
    return 4 * L + 14


def emulation_ops_per_unit(L, n1_table):
    """FP32 operations the split form spends on the same unit in double-float
    (an FMA counts two): L Horner or accumulation steps of 38, one complex
    double-float product of 50 and one complex double-float sum of 22; where
    the n1 recurrence runs (no per-record X(n1) table) each point also advances
    the prefactor and its ratio, another complex product of 50 and a
    complex-by-real one of 20.  A pipe-utilisation figure, not the method's work."""
    return 38 * L + (72 if n1_table > 0 else 142)


def walk_flops(info, ndens):
    """Algorithmic flops of one walk pass over all classes: the sum over classes
    L of records(L) x half-sphere points x (4L + 14), times the densities."""
    return ndens * sum(n * info["ng_half"] * method_flops_per_unit(L)
                       for L, n in enumerate(info["pairs_by_class"]))


def walk_emulation_ops(info, ndens):
    return ndens * sum(n * info["ng_half"] * emulation_ops_per_unit(L, info.get("n1_table", 0))
                       for L, n in enumerate(info["pairs_by_class"]))


def traffic_from_profile(kernel: str, workload: str):
    """dram bytes per walk pass from the committed ncu summary of this kernel
    and workload, if it was taken on the current kernel source (its recorded
    source hash must match)."""
    tag = {"diamond": "diamond240_k444", "molecular_crystal": "molecular_crystal"}[workload]
    path = os.path.join(ROOT, "profiles", f"{kernel}_{tag}.md")
    src_name = "tc.cu" if kernel.startswith("k_tc_") else ("walk_split.cu" if kernel.endswith("_split") else "walk.cu")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{16,64})", txt)
    t = re.search(r"dram_bytes_per_pass:\s*([0-9.eE+]+)", txt)
    if not m or not t:
        return None
    src = open(os.path.join(ROOT, "paper_2509_16460_gb300", "csrc", src_name), "rb").read()
    if hashlib.sha256(src).hexdigest()[:len(m.group(1))] != m.group(1):
        return None
    return float(t.group(1))


def omp_threads():
    threads = os.cpu_count() or 1
    try:
        import ctypes
        gomp = ctypes.CDLL("libgomp.so.1")
        threads = int(gomp.omp_get_max_threads())
    except OSError:
        pass
    return threads


def cpu_oracle_run(w, pair_stride):
    import oracle
    r = oracle.lrj(w, pair_stride=pair_stride, want_j0n=False, want_rho=False)
    units = r["units"] * w.ndens
    return r, units, omp_threads()


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


def make_workload(W, name):
    return {"molecular_crystal": W.cfg3, "diamond": W.cfg2}[name]()


# form -> (pipe, per-pair cutoff eps, contraction): "split_tc" is the split form with the
# tensor-core separable contraction of the structure-factor pass (orthorhombic cells)
FORMS = {"split_tc": ("split", 0.0, 1), "split": ("split", 0.0, 0), "fp64": ("fp64", 0.0, 0),
         "split_pair_gcut": ("split", PAIR_GCUT_EPS, 0), "fp64_pair_gcut": ("fp64", PAIR_GCUT_EPS, 0)}


def measured_bf16_peak():
    """Sustained dense bf16 rate of this machine's GB300 (measured file if
    present, else the recipe's fallback), for a kernel timed inside a long step."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["bf16_tflops_sustained"]) * 1e12, "MEASURED_PEAKS.json bf16_tflops_sustained, of measured"
    except (OSError, KeyError, ValueError):
        return 1.7e15, "fallback 1.7 PFLOP/s bf16 sustained, of fallback"


def measure_form(ctx, w, wname, form):
    """Times whole builds of one form on device buffers (CUDA events on the
    launching stream, L2 flushed between steps, clocks sampled), then end to end
    through the host-buffer entry point, and derives the roofline of the
    dominant walk from the library's per-phase events."""
    import numpy as np
    ftcj, torch, args, dist = ctx["ftcj"], ctx["torch"], ctx["args"], ctx["dist"]
    world, rank, local = ctx["world"], ctx["rank"], ctx["local"]
    flush, stream, barrier = ctx["flush"], ctx["stream"], ctx["barrier"]
    pipe, eps, contraction = FORMS[form]
    prec = ftcj.FTCJ_PREC_SPLIT if pipe == "split" else ftcj.FTCJ_PREC_FP64
    sharded = world > 1
    plan = ftcj.Plan.from_workload(w, precision=prec, pair_gcut_eps=eps, contraction=contraction,
                                   shard_count=world if sharded else 0, shard_index=rank if sharded else 0)
    info = plan.info
    Dk = ctx["Dk"]
    nd = w.ndens
    Jk = torch.empty_like(Dk)
    EJ = torch.empty(nd, dtype=torch.float64, device="cuda")
    # the units of the whole build: a shard plan counts its own share
    units = float(info["pair_g_units"]) * nd
    if sharded:
        t = torch.tensor([units], dtype=torch.float64, device="cuda")
        dist.all_reduce(t)
        units = float(t.item())
    walk_ev = []

    def step():
        if not sharded:
            plan.jbuild(Dk, Jk, EJ)
            return
        # the record-sharded build (ftcj.sharded_jbuild's steps), with events
        # around the rho step (a3 + a4) for the roofline
        for b0 in range(0, nd, plan.max_dens):
            b1 = min(nd, b0 + plan.max_dens)
            D0n = plan.fold_density(Dk[b0:b1].contiguous())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rho = plan.rho(D0n)
            e1.record(stream)
            walk_ev.append((e0, e1))
            dist.all_reduce(torch.view_as_real(rho))
            Wg, E = plan.potential(rho)
            J0n = plan.jback(Wg)
            dist.all_reduce(J0n)
            Jk[b0:b1] = plan.unfold_j(J0n)
            EJ[b0:b1] = E

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    walk_ev.clear()
    if not sharded:
        plan.profile_enable(args.steps)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(statistics.mean(step_ms), dist, "cuda")
    value = strong_rate(units, ms * 1e-3)
    # roofline of the dominant walk pass
    walked = info["pair_g_units_walked"] / info["pair_g_units"] if info["pair_g_units"] else 1.0
    flops = walk_flops(info, nd) * walked
    emu = walk_emulation_ops(info, nd) * walked
    suffix = "_split" if pipe == "split" else ""
    if not sharded:
        phase_ms, batches, launches = plan.profile_read()
        plan.profile_enable(0)
        rho_name = "k_tc_rho" if contraction else "k_rho_walk" + suffix
        j_name = "k_tc_j" if info["j_contraction"] else "k_j_walk" + suffix
        walks = {rho_name: phase_ms["rho_walk"], j_name: phase_ms["j_walk"]}
        kname = max(walks, key=walks.get)
        pass_ms = walks[kname] * max(1, -(-nd // plan.max_dens)) / max(batches, 1)
        rho_pass_ms = phase_ms["rho_walk"] * max(1, -(-nd // plan.max_dens)) / max(batches, 1)
        j_pass_ms = phase_ms["j_walk"] * max(1, -(-nd // plan.max_dens)) / max(batches, 1)
        phases = {k: v / max(batches, 1) for k, v in phase_ms.items()}
        timed_what = "the library's phase events around the whole walk pass (all class-part launches)"
    else:
        kname = "k_hermite_map" + ("_df" if pipe == "split" else "") + " + k_rho_walk" + suffix
        pass_ms = statistics.mean(a.elapsed_time(b) for a, b in walk_ev) * len(walk_ev) / args.steps
        phases = None
        launches = plan.launches_per_batch() * args.steps * max(1, -(-nd // plan.max_dens))
        timed_what = "CUDA events around the rho step (Hermite map + structure-factor walk) of this rank's share"
    achieved = flops / (pass_ms * 1e-3)
    peak = ctx["peaks"][pipe]
    parts = info["rho_walk_launches"] if "rho" in kname else info["j_walk_launches"]
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic_from_profile(kname, wname) if (eps == 0 and not sharded) else None,
                "kernel": kname, "launches_per_pass": parts,
                "pipe": "FP64" if pipe == "fp64" else "FP32",
                "peak_source": f"measured {'FP64' if pipe == 'fp64' else 'FP32'} FMA throughput "
                               "(ftcj_probe_fma_peak) on this GPU, of measured",
                "flops_rule": "per pass: sum over classes L of records(L) x half-sphere points x (4L+14), "
                              "x densities" + (" x walked fraction of the units" if eps > 0 else ""),
                "flops_per_pass": flops, "pass_ms": pass_ms, "timed": timed_what,
                "nominal_peak": 152 * 2 * 2.07e9 * (2 if pipe == "fp64" else 128) / 1e12}
    if contraction and not sharded:
        # the tensor-core passes: bf16 MMA flops (slice products included) against the sustained dense
        # bf16 rate, and their algorithmic (4L+14) rate; the dominant one heads the roofline
        bf16_peak, bf16_src = measured_bf16_peak()
        reps = max(1, -(-nd // plan.max_dens))
        tc = {}
        for key, kern, mma, t_ms, note in (
                ("tc_rho", "k_tc_rho", float(info["tc_mma_flops"]) * reps, rho_pass_ms,
                 "21 bf16 slice products per product exact to 2^-41 (6 slices a side), real form of the "
                 "complex product (4 real per complex multiply-add)"),
                ("tc_j", "k_tc_j", float(info["tc_j_mma_flops"]) * reps, j_pass_ms,
                 "28 bf16 slice products per product exact to 2^-45 (7 slices a side), real form of the "
                 "complex product")):
            if mma <= 0:
                continue
            tc[kern] = {"bound": "tensor", "kernel": kern, "pass_ms": t_ms,
                        "achieved": mma / (t_ms * 1e-3) / 1e12, "peak": bf16_peak / 1e12, "unit": "TFLOP/s",
                        "frac": mma / (t_ms * 1e-3) / bf16_peak, "mma_flops_per_pass": mma,
                        "peak_source": bf16_src,
                        "algorithmic_tflops": walk_flops(info, nd) / (t_ms * 1e-3) / 1e12,
                        "algorithmic_frac_of_fp32": walk_flops(info, nd) / (t_ms * 1e-3) / peak,
                        "traffic": traffic_from_profile(kern, wname), "note": note}
            roofline[key] = tc[kern]
        if kname in tc:
            head = dict(tc[kname])
            head["launches_per_pass"] = parts
            head["timed"] = timed_what
            head["flops_rule"] = ("per pass: the bf16 MMA flops the kernel issues (every slice product and "
                                  "padding column, 2 per multiply-add), x density groups")
            for k2 in ("tc_rho", "tc_j"):
                if k2 in roofline:
                    head[k2] = roofline[k2]
            head["alu_view"] = {k2: roofline[k2] for k2 in ("achieved", "peak", "frac", "pipe") if k2 in roofline}
            roofline = head
    if pipe == "split":
        roofline["fp32_pipe_ops_per_pass"] = emu
        roofline["fp32_pipe_ops_frac"] = emu / (pass_ms * 1e-3) / peak
        roofline["fp32_pipe_ops_note"] = ("double-float emulation operations (38L+72 with the X(n1) table, "
                                          "38L+142 without) per unit: pipe utilisation, not the method's work")
        roofline["fp64_equivalent_vs_fp64_peak"] = achieved / ctx["peaks"]["fp64"]
    out = {"value": value, "unit": UNIT, "ms_per_step": ms, "step_ms_min": min(step_ms),
           "roofline": roofline, "gpu_launches": int(launches), "clocks": clocks, "wall_s_timed_region": t_wall,
           "phase_ms_per_step": phases, "pair_g_units_per_step": units,
           "walk_shape": {"rho_blocks": info["rho_blocks"], "n1_table": info["n1_table"],
                          "nchunks": info["nchunks"], "launches_per_batch": plan.launches_per_batch()}}
    if eps > 0:
        out["pair_gcut_eps"] = eps
        out["walked_fraction_of_units"] = walked
        out["screened_fraction_of_units"] = info["pair_g_units_screened"] / info["pair_g_units"]
    # end to end: pinned host D^k in, J^k and E_J out, copies inside the timed region
    Dk_h = ctx["Dk_host"]
    Jk_h = torch.empty(Dk_h.shape, dtype=torch.complex128).pin_memory()
    EJ_h = torch.empty(nd, dtype=torch.float64).pin_memory()

    def e2e_step():
        if not sharded:
            plan.jbuild_host(Dk_h, Jk_h, EJ_h)
            return
        Dd = Dk_h.to("cuda", non_blocking=True)
        J, E = ftcj.sharded_jbuild(plan, Dd)
        Jk_h.copy_(J, non_blocking=True)
        EJ_h.copy_(E, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step()
    e2e_t = []
    barrier()
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.mean(e2e_t), dist, "cuda")
    out["e2e"] = {"value": strong_rate(units, e2e_s), "unit": UNIT, "ms_per_step": e2e_s * 1e3,
                  "h2d_bytes_per_step": Dk_h.numel() * 16,
                  "d2h_bytes_per_step": Jk_h.numel() * 16 + EJ_h.numel() * 8,
                  "transfer": ("pinned host buffers read and written by the device over the host link (the split "
                               "form's fold reads only the upper triangle of the Hermitian D^k)") if not sharded else
                              "pinned host D^k copied in, J^k and E_J copied out, around the sharded build"}
    out["result"] = (Jk.cpu().numpy(), EJ.cpu().numpy())
    out["info"] = info
    plan.close()
    return out


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
    # the persistent form: every cell's walks, potentials and energies in one launch over a work queue
    t0 = time.perf_counter()
    BP = ftcj.Batch(cells, precision=ftcj.FTCJ_PREC_SPLIT, persistent=True)
    setup_p = time.perf_counter() - t0
    units_p = sum(float(i["pair_g_units"]) * w.ndens for i, w in zip(BP.infos, cells))
    Jp, Ep = BP.outputs_like(Dks)
    torch.cuda.synchronize()
    BP.capture(Dks, Jp, Ep, stream=s)
    for _ in range(3):
        BP.replay(stream=s)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        ms_p = time_events(lambda: BP.replay(stream=s), steps, flush, s)
    out["persistent_graph_replay"] = {"ms_per_step": ms_p, "value": units_p / (ms_p * 1e-3), "unit": UNIT,
                                      "setup_s": setup_p, "status": BP.status(stream=s),
                                      "note": "default walk shapes; walks, potentials and energies of all cells "
                                              "in one persistent launch, transforms and maps per cell on streams"}
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
    out["max_abs_dJ_persistent_vs_serial"] = max(float((a - b[0]).abs().max()) for a, b in zip(Jp, outs))
    for p in plans:
        p.close()
    B.close()
    BP.close()
    return out


def autotune_leg(ftcj, W, torch, flush, steps):
    """The headline cell's split build with the walk shape the autotuner picks."""
    import numpy as np
    w = W.cfg3()
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    chunk, rb, _ = ftcj.autotune(w, precision=ftcj.FTCJ_PREC_SPLIT)
    tune_s = time.perf_counter() - t0
    p = ftcj.Plan.from_workload(w, precision=ftcj.FTCJ_PREC_SPLIT, chunk_points=chunk, rho_blocks=rb)
    units = float(p.info["pair_g_units"]) * w.ndens
    J, E = p.jbuild(Dk)
    for _ in range(2):
        p.jbuild(Dk, J, E)
    ms = time_events(lambda: p.jbuild(Dk, J, E), steps, flush, stream)
    p.close()
    return {"ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT, "chunk_points": chunk,
            "rho_blocks": rb, "shape_note": "0 = the plan's own default", "autotune_s": tune_s}


def diamond_leg(ctx, forms=("split_tc", "split", "fp64")):
    """Secondary line: the diamond-like 240-AO cell, k 4x4x4, every form timed
    as the headline is, and (unless disabled) checked whole against the oracle."""
    import numpy as np
    W, torch = ctx["W"], ctx["torch"]
    w = W.cfg2()
    sub = dict(ctx)
    sub["Dk"] = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    sub["Dk_host"] = torch.from_numpy(np.ascontiguousarray(w.Dk)).pin_memory()
    out = {"workload": WORKLOADS["diamond"]}
    res = {}
    for f in forms:
        r = measure_form(sub, w, "diamond", f)
        res[f] = r.pop("result")
        info = r.pop("info")
        out[f] = r
    out["pair_g_units_per_step"] = float(info["pair_g_units"]) * w.ndens
    if not ctx["args"].no_cpu_baseline:
        t0 = time.perf_counter()
        ref, cu, threads = cpu_oracle_run(w, 1)
        out["cpu_oracle_whole_build"] = {"value": cu / ref["seconds"], "unit": UNIT, "cores": threads,
                                         "seconds": ref["seconds"], "wall_s": time.perf_counter() - t0}
        for f, (Jg, Eg) in res.items():
            out[f]["max_abs_dJ_vs_oracle"] = float(np.abs(Jg - ref["Jk"]).max())
            out[f]["abs_dEJ_vs_oracle"] = float(np.abs(Eg - ref["EJ"]).max())
    return out


def slab_leg(ftcj, W, torch, flush, steps):
    """The surface slab (rock-salt 2x2 (001), 4 layers + CO, 940 AOs, k 3x3x1):
    split and FP64 builds, and the split plan's nuclear gradient (dE_J/dR of
    every centre)."""
    import numpy as np
    w = W.cfg5()
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    out = {"workload": "rock-salt (001) 2x2 slab, 4 layers (16 Mg-like + 16 O-like) + CO, 20 bohr vacuum, "
                       f"{len(w.xyz)} centres, {w.nao} spherical AOs, k 3x3x1, omega 0.4", "ndens": w.ndens}
    stream = torch.cuda.current_stream()
    res = {}
    for form, prec, con in (("split_tc", ftcj.FTCJ_PREC_SPLIT, ftcj.FTCJ_CONTRACT_TC),
                            ("split", ftcj.FTCJ_PREC_SPLIT, ftcj.FTCJ_CONTRACT_WALK),
                            ("fp64", ftcj.FTCJ_PREC_FP64, ftcj.FTCJ_CONTRACT_WALK)):
        p = ftcj.Plan.from_workload(w, precision=prec, contraction=con)
        units = float(p.info["pair_g_units"]) * w.ndens
        out["pair_g_units_per_step"] = units
        J, E = p.jbuild(Dk)
        for _ in range(2):
            p.jbuild(Dk, J, E)
        ms = time_events(lambda: p.jbuild(Dk, J, E), steps, flush, stream)
        out[form] = {"ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT}
        if con == ftcj.FTCJ_CONTRACT_TC:
            out[form]["status"] = p.status()
            out[form]["j_contraction"] = int(p.info["j_contraction"])
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
    out["split_tc_vs_fp64_max_abs_dJ"] = float((res["split_tc"][0] - res["fp64"][0]).abs().max())
    out["split_tc_vs_fp64_abs_dEJ"] = float((res["split_tc"][1] - res["fp64"][1]).abs().max())
    return out


def gpw_leg(ctx, forms=("split_tc", "fp64")):
    """The molecular crystal with the compact/diffuse classification (Sec. 2.6):
    the default alpha_cut = w^2/2 = 0.125 makes the 0.1 s exponent of every
    centre diffuse, and the s-s pairs of those primitives (with their lattice
    images) take the GPW route (App. E): collocation on the real-space grid,
    the separable transform onto the sphere, the full-range potential and the
    adjoint integration, all FP64.  The classified build is a different
    Coulomb operator from the long-range headline (every integral touching a
    DD density takes the full-range kernel), so its time is context for the
    route, not a comparison."""
    import numpy as np
    ftcj, torch, W = ctx["ftcj"], ctx["torch"], ctx["W"]
    flush, stream = ctx["flush"], ctx["stream"]
    steps = max(3, min(ctx["args"].steps, 10))
    w = W.cfg3()
    Dk = ctx["Dk"]
    out = {"workload": WORKLOADS[HEADLINE] + ", compact/diffuse classified (alpha_cut = w^2/2)",
           "ndens": w.ndens}
    res = {}
    for form in forms:
        pipe, _, con = FORMS[form]
        prec = ftcj.FTCJ_PREC_SPLIT if pipe == "split" else ftcj.FTCJ_PREC_FP64
        p = ftcj.Plan.from_workload(w, precision=prec, contraction=con, classify=True)
        info = p.info
        units = float(info["npairs_ordered"] + info["dd_pairs_ordered"]) * info["ng_full"] * w.ndens
        J, E = p.jbuild(Dk)
        for _ in range(2):
            p.jbuild(Dk, J, E)
        torch.cuda.synchronize()
        p.profile_enable(steps)
        ms = time_events(lambda: p.jbuild(Dk, J, E), steps, flush, stream)
        phase_ms, batches, launches = p.profile_read()
        p.profile_enable(0)
        ph = {k: v / max(batches, 1) for k, v in phase_ms.items()}
        npts = float(np.prod(info["gpw_grid"]))
        # collocation and integration: 2 (L + 1) flops per DD record, grid point and density each
        flops = sum(2.0 * (c + 1) * n for c, n in enumerate(info["dd_pairs_by_class"])) * npts * w.ndens * 2
        gpw_ms = ph["gpw_rho"] + ph["gpw_j"]
        # the split form runs the two grid contractions in double-float on the FP32 pipe
        dfp = info["gpw_separable"] == 2
        peak = ctx["peaks"]["split" if dfp else "fp64"]
        r = {"ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT,
             "dd_records": info["dd_pairs"], "dd_ordered_pairs": info["dd_pairs_ordered"],
             "dd_records_by_class": info["dd_pairs_by_class"], "compact_records": info["npairs"],
             "alpha_cut": info["alpha_cut"], "gpw_grid": info["gpw_grid"], "gpw_separable": info["gpw_separable"],
             "gpw_launches": info["gpw_launches"], "phase_ms_per_step": ph, "gpw_ms_per_step": gpw_ms,
             "gpw_share": gpw_ms / ms,
             "gpw_roofline": {"bound": "alu", "pipe": "fp32 (double-float)" if dfp else "fp64",
                              "achieved": flops / (gpw_ms * 1e-3) * 1e-12,
                              "peak": peak * 1e-12, "unit": "TFLOP/s",
                              "frac": flops / (gpw_ms * 1e-3) / peak,
                              "flops_per_step": flops,
                              "note": "algorithmic flops of the collocation and integration contractions over "
                                      "the time of both GPW phases (their reduction, six transform passes and "
                                      "row sums included); peak: the FMA probe of this run for the pipe the "
                                      "contractions run on (FP64, or FP32 for double-float), measured"}}
        if con == ftcj.FTCJ_CONTRACT_TC:
            r["status"] = p.status()
        out[form] = r
        res[form] = (J.clone(), E.clone())
        p.close()
    if "fp64" in res:
        for f in res:
            if f != "fp64":
                out[f]["max_abs_dJ_vs_fp64"] = float((res[f][0] - res["fp64"][0]).abs().max())
                out[f]["abs_dEJ_vs_fp64"] = float((res[f][1] - res["fp64"][1]).abs().max())
    return out


def run_reference(args, world, rank):
    """The reference arm is the CPU oracle, timed as it stands on the host
    cores, on a bounded sample of the headline workload per step (every
    REFERENCE_STRIDE-th ordered screened pair over the whole G sphere, with the
    k-mesh transforms of the whole density): same metric and unit."""
    if rank != 0:
        return 0
    import oracle
    from paper_2509_16460_gb300 import workloads as W
    oracle.build()
    w = W.cfg3()
    stride = REFERENCE_STRIDE
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
    sample = (f"every {stride}th ordered screened primitive pair of the workload over the full G sphere "
              f"({units:.3e} pair*G units per step), both densities, whole k-mesh transforms")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[HEADLINE], "form": "fp64 CPU oracle", "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
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
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    peaks = {"fp64": ftcj.probe_fma_peak(0), "split": ftcj.probe_fma_peak(1)}
    ctx = dict(ftcj=ftcj, torch=torch, W=W, args=args, dist=dist, world=world, rank=rank, local=local,
               flush=flush, stream=torch.cuda.current_stream(), barrier=barrier, peaks=peaks)
    if args.leg:
        steps = max(3, min(args.steps, 10))
        if args.leg == "diamond":
            out = diamond_leg(ctx)
            for f in ("split_tc", "split", "fp64"):
                out[f].pop("clocks", None)
        elif args.leg == "batch":
            out = batch_leg(ftcj, W, torch, flush, steps)
        elif args.leg == "slab":
            out = slab_leg(ftcj, W, torch, flush, steps)
        elif args.leg == "gpw":
            w3 = W.cfg3()
            ctx["Dk"] = torch.from_numpy(np.ascontiguousarray(w3.Dk)).cuda()
            out = gpw_leg(ctx)
        else:
            out = autotune_leg(ftcj, W, torch, flush, steps)
        print(json.dumps({"leg": args.leg, **out}), flush=True)
        return 0

    w = W.cfg3()
    ctx["Dk"] = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    ctx["Dk_host"] = torch.from_numpy(np.ascontiguousarray(w.Dk)).pin_memory()
    ortho = bool(np.allclose(w.A - np.diag(np.diag(w.A)), 0.0))
    head_form = "split_tc" if ortho else "split"
    want = [head_form] + [f for f in args.forms.split(",") if f and f != head_form]
    forms, results, infos = {}, {}, {}
    for f in want:
        if f not in FORMS:
            raise SystemExit(f"unknown form {f}")
        r = measure_form(ctx, w, HEADLINE, f)
        results[f] = r.pop("result")
        infos[f] = r.pop("info")
        forms[f] = r
    head = forms[head_form]
    info = infos[head_form]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None,
        "dtype": ("bf16-sliced tcgen05 contractions (structure factor: 6 slices a side; back-contraction: "
                  "7 slices a side where the plan takes it, else the f32x2 walk) with exact FP32 level sums, "
                  "f32x2 (double-float) operands and window sums, f64 setup/sums/E_J"
                  if head_form == "split_tc" else "f32x2 walks (double-float), f64 setup/sums/E_J"),
        "data": "synthetic",
        "config": {"workload": WORKLOADS[HEADLINE], "form": head_form, "ndens": w.ndens,
                   "pair_g_units_per_step": head["pair_g_units_per_step"],
                   "npairs_ordered": info["npairs_ordered"] if world == 1 else None,
                   "pair_records": info["npairs"] if world == 1 else None,
                   "ng_full": info["ng_full"], "nao": info["nao"], "nk": info["nk"],
                   "records_by_class": info["pairs_by_class"] if world == 1 else None,
                   "rho_blocks": info["rho_blocks"], "n1_table": info["n1_table"],
                   "l2": f"{L2_FLUSH_BYTES >> 20} MB buffer written between timed steps (inputs of "
                         f"{w.Dk.nbytes >> 20} MB also exceed the 129 MB L2)",
                   "parallelism": (f"{world} GPUs, pair records sharded, NCCL all-reduce of rho(G) and J^0n"
                                   if world > 1 else "1 GPU")},
        "e2e": {k: head["e2e"][k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")},
        "gpu_launches": head["gpu_launches"],
        "roofline": head["roofline"],
        "clocks": head["clocks"],
        "forms": forms,
    }
    if "fp64" in forms:
        line["split_speedup_vs_fp64"] = forms["fp64"]["ms_per_step"] / head["ms_per_step"]
        for f in forms:
            if f != "fp64":
                forms[f]["max_abs_dJ_vs_fp64"] = float(np.abs(results[f][0] - results["fp64"][0]).max())
                forms[f]["abs_dEJ_vs_fp64"] = float(np.abs(results[f][1] - results["fp64"][1]).max())
        line["split_vs_fp64_max_abs_dJ"] = forms[head_form]["max_abs_dJ_vs_fp64"]
        line["split_vs_fp64_abs_dEJ"] = forms[head_form]["abs_dEJ_vs_fp64"]
    if rank == 0 and world == 1 and not args.no_extra:
        extra_steps = max(3, min(args.steps, 10))
        line["diamond"] = diamond_leg(ctx)
        line["batch"] = batch_leg(ftcj, W, torch, flush, extra_steps)
        line["gpw"] = gpw_leg(ctx)
        line["workloads"] = {"slab": slab_leg(ftcj, W, torch, flush, extra_steps),
                             "molecular_crystal_autotuned": autotune_leg(ftcj, W, torch, flush, extra_steps)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle as it stands on the host cores, on a bounded pair sample of the headline workload
        stride = CPU_BASELINE_STRIDE
        r, cu, threads = cpu_oracle_run(w, stride)
        line["cpu_baseline"] = {
            "value": cu / r["seconds"], "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"every {stride}th ordered screened primitive pair ({r['npairs']} of "
                       f"{info['npairs_ordered']}) over the full sphere of {r['nG']} G, both densities, with the "
                       "whole k-mesh transforms of the build (not scaled down), one run"),
            "seconds": r["seconds"], "pair_g_units_in_sample": cu}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
