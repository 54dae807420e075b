"""Throughput of the cumulant-LBM tree-drag step on GB300.

One step = one coarse step of the whole path: collide-stream of every level
(2^l sub-steps of level l), faces, bounce-back with the FP64 drag reduction,
and the refinement-interface transfer, replayed as one CUDA graph.  Before
the warm-up each domain is autotuned (collide-kernel variants and z splits,
timed by the library itself) and then re-initialised to the impulsive start,
so the timed steps run the measured-fastest schedule on the usual state.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is whole-job MLUPS (cell updates summed over
levels, level l counted 2^l times per coarse step, over all ranks) with the
state resident in HBM; ``e2e`` is the same metric through the C-ABI including
binding (table upload and initialisation) and a host read of the drag after
every step.  With N > 1 every rank runs an independent replica (the problem
does not shard on one GPU per rank here) and the time is the maximum over
ranks.  ``--impl reference`` times the FP64 CPU oracle on the host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CASE = "amr2"
QUARTER = "amr2_quarter"  # the same tree case scaled down 4x per axis, for the C_D comparison
PRECISION_CASE = "amr4"
BYTES_PER_UPDATE = 2 * 27 * 4  # read and write 27 FP32 populations
NOMINAL_HBM_GBS = 7900.0  # GB300's nominal HBM3e bandwidth (the measured copy peak is the roofline)
KERNEL_SOURCES = ["paper_2603_27954_gb300/csrc/collide.cuh", "paper_2603_27954_gb300/csrc/cumulant.cuh"]


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def profiled_traffic():
    """DRAM bytes per collide launch from the committed ncu summary, if it was
    taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "collide_amr2_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    if d.get("kernel_hash") != kernel_hash():
        return None
    return d


def job_rate(units_per_rank, steps, ms_local, world, reduce_max):
    """Whole-job rate over all ranks: every rank's units over the slowest
    rank's time (max over ranks), in millions per second; also that time."""
    ms_max = reduce_max(ms_local)
    return units_per_rank * world * steps / (ms_max / 1e3) / 1e6, ms_max


def workload_desc(L, W, case, precision=None):
    c = W.CASES[case]
    desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                         re_h=c["re_h"], precision=precision or L.LBM_FP32)
    return desc, L.tree_desc(**c["tree"]), c


def tune(L, dom, u_in, steps):
    """Autotune the domain's schedule, then restore the impulsive start (the
    tuner advances the flow) with fresh force sums."""
    import numpy as np
    best, _ = dom.autotune(steps)
    L.lbm_init_uniform(dom.h, 1.0, np.array([u_in, 0.0, 0.0]))
    L.lbm_reset_force(dom.h)
    return dict(best.as_dict(), overlap_features=dom.get_overlap_features())


def fixed_schedule(dom, spec):
    """odd,even,z_even,z_odd[,overlap feature mask]: a fixed schedule (for
    profiling the kernels a tuned run chose)."""
    v = [int(x) for x in spec.split(",")]
    dom.set_schedule(0, *v[:4])
    if len(v) > 4:
        dom.set_overlap_features(v[4])
    return dict(dom.get_schedule().as_dict(), overlap_features=dom.get_overlap_features())


def measure_form(L, W, torch, stream, case, precision, steps, warmup, timing_steps=20, tune_steps=3, schedule=None):
    """Whole-path MLUPS of one workload in one storage form (CUDA events on
    the domain's stream) under its autotuned schedule, the collide kernels'
    algorithmic GB/s from the library's per-class timing, and the C_D after
    the timed steps."""
    desc, tree, c = workload_desc(L, W, case, precision)
    dom = L.Domain(desc, tree=tree, stream=stream)
    updates, _ = dom.work_per_step()
    if schedule:
        schedule = fixed_schedule(dom, schedule)
    else:
        schedule = tune(L, dom, c["u_in"], tune_steps)
    dom.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dom.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    dom.set_timing(True)
    dom.step(timing_steps)
    kms, _, kunits = dom.get_timing()
    dom.set_timing(False)
    bpu = 108 if precision == L.LBM_FP16_DEV else BYTES_PER_UPDATE
    gbs = (kunits[0] + kunits[1]) * bpu / ((kms[0] + kms[1]) / 1e3) / 1e9
    _, _, cd = dom.drag()
    cells = sum(L.lbm_level_info(dom.h, l)["n_fluid"] for l in range(desc.levels))
    gb = dom.nbytes / 1e9
    dom.close()
    torch.cuda.empty_cache()
    return {"value": updates * steps / (ms / 1e3) / 1e6, "ms_per_step": ms / steps, "collide_gbs": gbs,
            "bytes_per_update": bpu, "cd": cd, "updates_per_step": updates, "cells": cells, "device_gb": gb,
            "schedule": schedule}


def fp16_form(L, W, torch, stream, steps, warmup, fp32_value, peak, schedule=None):
    """The FP16-deviation storage form on the same workload: MLUPS, its
    collide roofline at 108 B per update, and the speed-up over FP32."""
    r = measure_form(L, W, torch, stream, CASE, L.LBM_FP16_DEV, steps, warmup, tune_steps=8, schedule=schedule)
    return {"value": r["value"], "unit": "MLUPS", "speedup_vs_fp32": r["value"] / fp32_value,
            "ms_per_step": r["ms_per_step"],
            "dtype": "f16 storage of (f - f^eq(1, U e_x)) * 2^13, f32 collision, f64 reductions",
            "roofline": {"bound": "hbm", "achieved": r["collide_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": r["collide_gbs"] / peak, "bytes_per_update": 108}, "cd": r["cd"],
            "schedule": r["schedule"]}


def precision_form(L, W, torch, stream, steps, warmup, peak):
    """The four-level precision-form workload (about 6e8 active cells) in
    FP32 and FP16-deviation storage."""
    c = W.CASES[PRECISION_CASE]
    out = {"workload": "four-level tree drag: coarse %dx%dx%d in %d^3 blocks, L-system n=%d x %d children, "
                       "trunk %d finest cells, Re_H=%g, U=%g" % (*c["n0"], c["block"], c["tree"]["n"],
                                                                c["tree"]["children"], c["tree"]["trunk_cells"],
                                                                c["re_h"], c["u_in"]),
           "steps": steps, "warmup": warmup, "unit": "MLUPS"}
    for name, prec in (("fp32", L.LBM_FP32), ("fp16", L.LBM_FP16_DEV)):
        r = measure_form(L, W, torch, stream, PRECISION_CASE, prec, steps, warmup, timing_steps=2, tune_steps=1)
        out[name] = {"value": r["value"], "ms_per_step": r["ms_per_step"], "cd": r["cd"], "schedule": r["schedule"],
                     "roofline": {"bound": "hbm", "achieved": r["collide_gbs"], "peak": peak, "unit": "GB/s",
                                  "frac": r["collide_gbs"] / peak, "bytes_per_update": r["bytes_per_update"]},
                     "device_gb": r["device_gb"]}
        out["cells"] = r["cells"]
        out["updates_per_step"] = r["updates_per_step"]
    out["speedup_fp16_vs_fp32"] = out["fp16"]["value"] / out["fp32"]["value"]
    out["cd_rel_diff_fp16_vs_fp32"] = abs(out["fp16"]["cd"] - out["fp32"]["cd"]) / abs(out["fp32"]["cd"])
    return out


def batched_form(L, W, torch, stream, steps, peak, blocks=(16, 8)):
    """The 16-case batched form: the batch (one persistent collide launch per
    level depth and sub-step, one graph per coarse step) against the cases
    stepped one after another, each by its own CUDA graph, under the same
    kernel variants and z splits.  The tuner picks the block size (the cases
    built in 16^3 and in 8^3 blocks) and, per block size, the batch schedule
    (lbm_batch_autotune)."""
    per_block = {}
    for bsz in blocks:
        doms, updates = [], 0
        for c in W.batch_cases():
            desc = L.domain_desc(*c["n0"], levels=c["levels"], block=bsz, bc=c["bc"], u_in=c["u_in"],
                                 re_h=c["re_h"], i_u=c["i_u"], seed=c["seed"])
            d = L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)
            updates += d.work_per_step()[0]
            doms.append(d)
        nblocks = [L.lbm_level_info(d.h, 0)["n_active_blocks"] for d in doms]

        def timed(fn):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        def sequential(n):
            for _ in range(n):
                for d in doms:
                    d.step(1)

        batch = L.Batch(doms, stream=stream)
        best, tune_ms = batch.autotune(steps=3)
        batch.step(3)
        ms_batch = timed(lambda: batch.step(steps))
        batch.close()
        # the cases one after another under the same kernels and z splits
        for d in doms:
            d.set_schedule(0, best.odd_variant, best.even_variant, best.z_split_even, best.z_split_odd)
        sequential(3)
        ms_seq = timed(lambda: sequential(steps))
        gb = sum(d.nbytes for d in doms) / 1e9
        for d in doms:
            d.close()
        torch.cuda.empty_cache()
        per_block[bsz] = {"value": updates * steps / (ms_batch / 1e3) / 1e6,
                          "sequential_value": updates * steps / (ms_seq / 1e3) / 1e6,
                          "ms_per_step": ms_batch / steps, "sequential_ms_per_step": ms_seq / steps,
                          "updates_per_step": updates, "device_gb": gb, "schedule": best.as_dict(),
                          "autotune_ms_per_step": tune_ms, "coarse_blocks": [min(nblocks), max(nblocks)]}
    bsz = max(per_block, key=lambda k: per_block[k]["value"])
    r = per_block[bsz]
    return {"workload": "16 cases: trees of 1-4 child generations x Re_H {2.5e3, 1e4, 4e4, 1.2e5}, 2-3 levels, "
                        "I_u = 8 %% random-Fourier-mode inflow in half of them; block size picked by the tuner "
                        "(%d^3: %d-%d coarse blocks per case)" % (bsz, *r["coarse_blocks"]),
            "unit": "MLUPS", "steps": steps, "block": bsz, "updates_per_step": r["updates_per_step"],
            "device_gb": r["device_gb"], "value": r["value"], "sequential_value": r["sequential_value"],
            "speedup_vs_sequential": r["value"] / r["sequential_value"],
            "sequential": "the same cases one after another, each by its own CUDA graph (default reorderings), "
                          "under the batch's kernel variants and z splits",
            "ms_per_step": r["ms_per_step"],
            "sequential_ms_per_step": r["sequential_ms_per_step"], "schedule": r["schedule"],
            "autotune_ms_per_step": r["autotune_ms_per_step"],
            "path_frac": r["value"] * 1e6 * BYTES_PER_UPDATE / 1e9 / peak,
            "per_block_size": {str(k): {kk: v[kk] for kk in ("value", "sequential_value", "schedule")}
                               for k, v in per_block.items()}}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for ln in fh:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def oracle_case(case):
    """The oracle's simulation of a workload record, its cell updates per
    coarse step (level l counted 2^l times) and its geometry info."""
    import oracle as O
    from paper_2603_27954_gb300 import workloads as W
    c = W.CASES[case]
    t = c["tree"]
    tree = O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       azimuth_mode=t["azimuth_mode"], seed=t["seed"])
    sim, info = O.tree_case(*c["n0"], tree, t["trunk_cells"], c["re_h"], u_in=c["u_in"], levels=c["levels"],
                            block=c["block"], bc=c["bc"])
    updates = sum(int((sim.cell_type(l) == 0).sum()) << l for l in range(c["levels"]))
    return sim, updates, info, c


def oracle_timed(sim, steps, threads):
    """Wall time of `steps` oracle coarse steps on `threads` host threads."""
    import oracle as O
    prev = O.set_threads(threads)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    O.set_threads(prev)
    return dt


def oracle_sample(sim, updates, budget_s, threads, max_steps):
    """Time the oracle on a bounded sample of a workload: one coarse step to
    size it, then as many more (at least one, at most max_steps) as fit the
    budget; returns (MLUPS, steps timed, seconds)."""
    t1 = oracle_timed(sim, 1, threads)
    n = max(1, min(max_steps, int(budget_s / max(t1, 1e-3))))
    dt = oracle_timed(sim, n, threads)
    return updates * n / dt / 1e6, n, dt


METRIC = "D3Q27 cumulant LBM MLUPS & % HBM roofline; C_D rel. error vs FP64 oracle"


def workload_config(W):
    """The benchmark workload, identical in both arms."""
    c = W.CASES[CASE]
    return {"workload": "two-level tree drag: coarse %dx%dx%d in %d^3 blocks, L-system n=%d x %d children, trunk %g "
                        "finest cells, Re_H=%g, U=%g" % (*c["n0"], c["block"], c["tree"]["n"], c["tree"]["children"],
                                                         c["tree"]["trunk_cells"], c["re_h"], c["u_in"]),
            "l2": "no flush: the state (1.87 GB of populations and tables) is larger than the 129 MB L2"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # the FP64 oracle on the benchmark workload itself (the full two-level tree
    # case): one untimed coarse step, then full coarse steps, as many of the
    # requested --steps as fit about a minute of host time (a coarse step of
    # this workload takes seconds on the host)
    from paper_2603_27954_gb300 import workloads as W
    sim, updates, info, c = oracle_case(CASE)
    cores = os.cpu_count()
    oracle_timed(sim, min(args.warmup, 1), cores)
    mlups, n, dt = oracle_sample(sim, updates, 60.0, cores, args.steps)
    sample = ("%d full coarse steps of the benchmark workload (%d cell updates each, level l counted 2^l times) "
              "after %d untimed; --steps %d asked, capped at about a minute of host time" % (
                  n, updates, min(args.warmup, 1), args.steps))
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": n, "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": dt / n * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(W),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp16", action="store_true")
    ap.add_argument("--no-precision-form", action="store_true")
    ap.add_argument("--no-batched-form", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=20)
    ap.add_argument("--precision-steps", type=int, default=10)
    ap.add_argument("--timing-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--learned-form", type=float, default=0.0,
                    help="also run the learned form at this fraction of its full data set (1: ~1.9e5 branch samples, "
                         "about 16 GPU-minutes) and add its report")
    ap.add_argument("--cd-steps", type=int, default=300,
                    help="coarse steps of the scaled-down case for the C_D comparison with the oracle")
    ap.add_argument("--schedule", default=None,
                    help="odd,even,z_even,z_odd[,overlap mask]: fix the main workload's schedule instead of "
                         "autotuning it (for profiling the kernels a tuned run chose)")
    ap.add_argument("--fp16-schedule", default=None,
                    help="odd,even,z_even,z_odd[,overlap mask]: fix the FP16 form's schedule instead of autotuning it")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_2603_27954_gb300 import lbm as L
    from paper_2603_27954_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    desc, tree, c = workload_desc(L, W, CASE)
    stream = torch.cuda.Stream()
    dom = L.Domain(desc, tree=tree, stream=stream)
    if args.schedule:
        schedule = fixed_schedule(dom, args.schedule)
    else:
        # 8 timed steps per candidate: the z splits and reorderings differ by
        # a few per cent, about the noise of shorter samples
        schedule = tune(L, dom, c["u_in"], 8)
    # launches per coarse step under the schedule and reorderings chosen
    updates, kernels = dom.work_per_step()
    dom.step(args.warmup)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dom.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    value, ms_max = job_rate(updates, args.steps, ms, world, reduce_max)

    # cost of the FP64 interface ledger (on in the timed run): the same
    # schedule with the ledger off, timed the same way
    def time_steps(n):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dom.step(n)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    n_l = max(50, args.steps // 4)
    dom.set_interface_ledger(False)
    dom.step(3)
    ms_off = time_steps(n_l)
    dom.set_interface_ledger(True)
    dom.step(3)
    ms_on = time_steps(n_l)
    ledger = {"ms_per_step_on": ms_on, "ms_per_step_off": ms_off, "cost_frac": ms_on / ms_off - 1.0,
              "steps": n_l, "note": "FP64 interface ledger on (default, as in the timed run) against off, "
                                    "same tuned schedule"}

    # per-kernel timing with CUDA events on the domain's stream (direct launches)
    dom.set_timing(True)
    dom.step(args.timing_steps)
    kms, klaunch, kunits = dom.get_timing()
    dom.set_timing(False)
    peak, peak_kind = measured_peaks()
    coll_ms = kms[0] + kms[1]
    coll_units = kunits[0] + kunits[1]
    coll_launch = klaunch[0] + klaunch[1]
    coll_gbs = coll_units * BYTES_PER_UPDATE / (coll_ms / 1e3) / 1e9
    total_ms = float(kms.sum())
    tr = profiled_traffic()
    roofline = {"bound": "hbm", "kernel": "k_collide (fused collide-stream)",
                "achieved": coll_gbs, "peak": peak, "peak_kind": peak_kind + " copy bandwidth", "unit": "GB/s",
                "frac": coll_gbs / peak,
                "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": coll_gbs / NOMINAL_HBM_GBS,
                "traffic": tr["bytes_per_launch"] if tr else None,
                "traffic_note": tr["note"] if tr else "no ncu capture of the current kernel sources",
                "algorithmic_bytes_per_launch": coll_units * BYTES_PER_UPDATE / max(1, coll_launch),
                "even_gbs": kunits[0] * BYTES_PER_UPDATE / (kms[0] / 1e3) / 1e9 if kms[0] else None,
                "odd_gbs": kunits[1] * BYTES_PER_UPDATE / (kms[1] / 1e3) / 1e9 if kms[1] else None,
                "share_of_step_time": float(coll_ms / total_ms) if total_ms else None,
                "timed_launches": int(coll_launch),
                "path_frac": updates * BYTES_PER_UPDATE * args.steps / (ms_max / 1e3) / 1e9 / peak}

    # end to end through the C-ABI: re-bind (upload tables, initialise), then
    # every step followed by a host read of its drag (the copy of step k is
    # read while step k + 1 runs: two page-locked slots, one event each)
    torch.cuda.synchronize()
    # drag decomposition of the state the timed run reached (Sec. 3: C_D, C_F, C_P = C_D - C_F)
    _, _, cd_run = dom.drag()
    _, _, cf_run = dom.friction()
    steps_run = args.warmup + args.steps + args.timing_steps
    pop_bytes, uploaded = dom.memory_breakdown()
    slots = torch.zeros(2, 8, dtype=torch.float64, pin_memory=True)
    done = [torch.cuda.Event(), torch.cuda.Event()]
    barrier()
    h0 = time.perf_counter()
    L.lbm_bind_memory(dom.h, dom.buffer.data_ptr(), dom.buffer.numel())
    hb = time.perf_counter()
    for k in range(args.e2e_steps):
        dom.step(1)
        L.lbm_drag_enqueue(dom.h, slots[k % 2].data_ptr())
        done[k % 2].record(stream)
        if k > 0:
            done[(k - 1) % 2].synchronize()
            _, _, cd = L.lbm_drag_decode(dom.h, slots[(k - 1) % 2].numpy())
    done[(args.e2e_steps - 1) % 2].synchronize()
    _, _, cd = L.lbm_drag_decode(dom.h, slots[(args.e2e_steps - 1) % 2].numpy())
    torch.cuda.synchronize()
    h1 = time.perf_counter()
    e2e_value, _ = job_rate(updates, args.e2e_steps, (h1 - h0) * 1e3, world, reduce_max)
    info0 = L.lbm_level_info(dom.h, 0)
    geo = dom.geometry_info()

    fp16 = None
    if not args.no_fp16:
        fp16 = fp16_form(L, W, torch, stream, args.steps, args.warmup, value, peak, args.fp16_schedule)
    prec_form = None
    if not args.no_precision_form:
        prec_form = precision_form(L, W, torch, stream, args.precision_steps, 3, peak)
    batched = None
    if not args.no_batched_form:
        batched = batched_form(L, W, torch, stream, args.batched_steps, peak)

    learned = {"ran": False, "how": "bench.py --learned-form 1 (about 20 min: 1.9e5 LBM branch samples, "
                                     "two 4-member ensembles, eight held-out LBM judging runs)",
               "last_full_run": "profiles/learned_form_sectional_drag.md"}
    if args.learned_form > 0:
        from paper_2603_27954_gb300 import surrogate as SG
        counts = {k: max(1, int(round(v * args.learned_form))) for k, v in W.LEARNED_COUNTS.items()}
        learned, ens = SG.learned_form(stream=stream, counts=counts)
        for members in ens.values():
            for m in members:
                m.close()
        learned["scale"] = args.learned_form

    cpu = None
    cd_err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on bounded samples of the benchmark workload itself: full
        # coarse steps on all host cores (about 15 s) and one on a single core
        sim, o_upd, _, _ = oracle_case(CASE)
        cores = os.cpu_count()
        o_mlups, o_n, o_dt = oracle_sample(sim, o_upd, 15.0, cores, 50)
        one_dt = oracle_timed(sim, 1, 1)
        del sim
        cpu = {"value": o_mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": "%d full coarse steps (%.1f s) of the benchmark workload, %d cell updates per step" % (
                   o_n, o_dt, o_upd),
               "single_core": {"value": o_upd / one_dt / 1e6, "unit": "MLUPS", "cores": 1,
                               "sample": "1 full coarse step (%.1f s) of the benchmark workload" % one_dt}}
        # C_D of the GPU path against the oracle on the same tree case scaled
        # down 4x per axis (the oracle needs seconds per coarse step of the full case)
        qsim, q_upd, qinfo, qc = oracle_case(QUARTER)
        q_steps = args.cd_steps
        qsim.step(q_steps)
        import oracle as O
        q_last, _, _ = qsim.force()
        o_cd = O.drag_coefficient(q_last[0], qc["u_in"], qinfo["A_x"])
        del qsim
        out = {}
        for name, prec in (("fp32", L.LBM_FP32), ("fp16", L.LBM_FP16_DEV)):
            d2, t2, _ = workload_desc(L, W, QUARTER, prec)
            sdom = L.Domain(d2, tree=t2, stream=stream)
            sdom.step(q_steps)
            _, _, out[name] = sdom.drag()
            sdom.close()
        cd_err = {"case": "the benchmark's tree case scaled down 4x per axis (%s: coarse %dx%dx%d, n=%d x %d "
                          "children, trunk %g finest cells, Re_H=%g, 8^3 blocks), after %d coarse steps" % (
                              QUARTER, *qc["n0"], qc["tree"]["n"], qc["tree"]["children"], qc["tree"]["trunk_cells"],
                              qc["re_h"], q_steps),
                  "cd_gpu": out["fp32"], "cd_oracle": o_cd, "rel_err": abs(out["fp32"] - o_cd) / abs(o_cd),
                  "fp16_cd_gpu": out["fp16"], "fp16_rel_err": abs(out["fp16"] - o_cd) / abs(o_cd)}

    line = {
        "metric": METRIC,
        "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": workload_config(W),
        "workload_detail": {"finest_box": [list(L.lbm_level_info(dom.h, 1)["lo"]), list(L.lbm_level_info(dom.h, 1)["hi"])],
                            "cell_updates_per_step": updates,
                            "l2": "inputs larger than L2 (%.2f GB of populations and tables)" % (dom.nbytes / 1e9),
                            "replicas": world, "schedule": schedule},
        "roofline": roofline,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": uploaded / args.e2e_steps,
                "d2h_bytes_per_step": 64, "bind_ms": (hb - h0) * 1e3, "steps_ms": (h1 - hb) * 1e3,
                "note": "includes one binding (upload of %.1f MB of tables from pinned host memory, equilibrium "
                        "initialisation of %.2f GB of populations on the device) and a host read of the drag "
                        "(64 bytes, lbm_drag_enqueue into page-locked memory, read while the next step runs) of "
                        "each of %d steps; bytes per step = the upload over those steps" % (
                            uploaded / 1e6, pop_bytes / 1e9, args.e2e_steps)},
        "interface_ledger": ledger,
        "learned_form": learned,
        "precision_form": prec_form,
        "batched_form": batched,
        "gpu_launches": kernels * args.steps,
        "kernels_per_step": kernels,
        "cd": cd_run,
        "drag_decomposition": {"cd": cd_run, "cf": cf_run, "cp": cd_run - cf_run, "coarse_steps": steps_run},
        "cd_rel_err_vs_oracle": cd_err,
        "fp16_form": fp16,
        "cpu_baseline": cpu,
        "geometry": {"H_finest_cells": geo["H"], "A_x": geo["A_x"], "segments": geo["n_segments"],
                     "nu_finest": geo["nu_finest"], "fluid_cells_level0": info0["n_fluid"]},
    }
    dom.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
