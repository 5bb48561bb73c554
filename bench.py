"""Throughput of the correlation hot path on one GB300 (or N independent ranks).

Workload (focus refinement at paper scale): a 352x256x20 ensemble field with
n = 100 members (seeded synthetic stand-in for the paper's weather ensemble)
and two 32x32x20 regions (20,480 points each). One step runs the whole path
on the resident field:
  a1  ingest: per-point planes (FP64 stats, z-scores, ranks, sorted values)
  a3  all 419,430,400 cross pairs, Pearson, FP32, every value stored + extremes
  a4  the same for Spearman
  a12 2,000,000 seeded uniform cross pairs
  a6  KSG MI (k = 10) on them + extremes
  a5  16x16-bin histogram MI on them + extremes
The metric counts point-pair measure evaluations per second over the step
(2 x 419,430,400 + 2 x 2,000,000 per step); per-measure rates are reported
beside it. Multi-GPU (torchrun): every rank runs its own replica with its own
sampler stream (weak scaling); the only collective is the timing barrier and
max.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same step and scales it to the step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
from gen import configs  # noqa: E402

METRIC = "KSG-MI & Pearson point-pairs/s at M=100/1000 vs plain FP32 GPU, roofline %"
CFG = configs.FOCUS
N_ALL = 20480 * 20480
N_SAMPLED = CFG["sampled_pairs"]
PAIRS_PER_STEP = 2 * N_ALL + 2 * N_SAMPLED
N_SMS = 152
FP32_LANES = 128

# Algorithmic work per unit (stated in the design doc):
#   Pearson/Spearman all-pairs: 2n flops per pair (n multiply-adds).
#   KSG: n(n-1) Chebyshev distance evaluations + 2n(n-1) marginal comparisons
#        per pair (definition count), i.e. 3n(n-1) ALU operations.
#   ingest: read n*P*4 bytes, write planes 22 bytes per point-member + 16 per point.
ALG = {
    "allpairs_pearson": ("alu_flop", lambda n: 2.0 * n * N_ALL),
    "allpairs_spearman": ("alu_flop", lambda n: 2.0 * n * N_ALL),
    "ksg": ("alu_op", lambda n: 3.0 * n * (n - 1) * N_SAMPLED),
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return dict(hbm_gbs=d["hbm_gbs"], sm_max_mhz=d.get("sm_max_mhz", 2070.0),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_dev{device}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}",
                                          f"--query-gpu={self.Q}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                mx.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2309_03308_gb300 as pg
    from paper_2309_03308_gb300 import Params, build

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(dev)  # the library and the timing events share this stream
    torch.cuda.set_stream(stream)
    n = CFG["n"]
    if args.workload == "focus":
        F_host = gen.field(CFG["seed"], CFG["X"], CFG["Y"], CFG["Z"], CFG["n"])
    else:  # focus-regions: only the two boxes, as two fields (profiling case, ~0.2 GB)
        F_host = np.stack([gen.field(CFG["seed"], CFG["X"], CFG["Y"], CFG["Z"], n, box=b)
                           for b in (CFG["box_a"], CFG["box_b"])])
    F_dev = torch.from_numpy(F_host).to(dev)
    F_pin = torch.from_numpy(F_host).pin_memory()
    cc = pg.Context(local_rank, stream=stream.cuda_stream)
    if args.workload == "focus":
        fid = fid_b = cc.load_field(F_dev)
        ra, rb = cc.define_regions(fid, [CFG["box_a"], CFG["box_b"]])
    else:
        fid, fid_b = cc.load_field(F_dev[0]), cc.load_field(F_dev[1])
        (ra,) = cc.define_regions(fid, [(0, 0, 0, 32, 32, 20)])
        (rb,) = cc.define_regions(fid_b, [(0, 0, 0, 32, 32, 20)])
    vals_p = torch.empty((20480, 20480), device=dev)
    vals_s = torch.empty((20480, 20480), device=dev)
    pa = torch.empty(N_SAMPLED, dtype=torch.int32, device=dev)
    pb = torch.empty(N_SAMPLED, dtype=torch.int32, device=dev)
    ksg = torch.empty(N_SAMPLED, device=dev)
    hist = torch.empty(N_SAMPLED, device=dev)
    offs = np.array([0, N_SAMPLED], np.int64)
    p_pear, p_spear = Params(pg.CC_PEARSON), Params(pg.CC_SPEARMAN)
    p_ksg, p_hist = Params(pg.CC_MI_KSG, k=CFG["k"]), Params(pg.CC_MI_BINNED, bins=CFG["bins"])
    names = ["ingest", "allpairs_pearson", "allpairs_spearman", "sample", "ksg", "hist"]

    def step(i, ev=None, host=False):
        def mark(j):
            if ev is not None:
                ev[j].record(stream)
        mark(0)
        if args.workload == "focus":
            cc.update_field(fid, F_pin.numpy() if host else F_dev)  # host: H2D inside the call
        else:
            cc.update_field(fid, F_pin[0].numpy() if host else F_dev[0])
            cc.update_field(fid_b, F_pin[1].numpy() if host else F_dev[1])
        mark(1)
        rp = cc.all_pairs(ra, rb, p_pear, values=vals_p)
        mark(2)
        rs = cc.all_pairs(ra, rb, p_spear, values=vals_s)
        mark(3)
        cc.sample_pairs(ra, rb, CFG["sampler_seed"], N_SAMPLED, stream=rank * 1000003 + i,
                        pa=pa, pb=pb)
        mark(4)
        if args.workload == "focus":
            rk = cc.segment_extremes(fid, p_ksg, pa, pb, offs, values=ksg)
            mark(5)
            rh = cc.segment_extremes(fid, p_hist, pa, pb, offs, values=hist)
        else:
            rk = [cc.eval_pairs(fid, fid_b, p_ksg, pa, pb, out=ksg)]
            mark(5)
            rh = [cc.eval_pairs(fid, fid_b, p_hist, pa, pb, out=hist)]
        mark(6)
        if host:  # device -> host read of the step's results
            ksg_h = ksg.cpu()
            hist_h = hist.cpu()
            return rp, rs, rk, rh, ksg_h, hist_h
        return rp, rs, rk, rh

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return t.item()

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    barrier()

    # device-resident timed region
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
    launches0 = pg.launch_count()
    with Clocks(local_rank) as clk:
        torch.cuda.synchronize()
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            res = step(args.warmup + i, evs[i])
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = pg.launch_count() - launches0
    ms = t0.elapsed_time(t1)
    ms = max_over_ranks(ms)
    stage_ms = {nm: statistics.median([evs[i][j].elapsed_time(evs[i][j + 1])
                                       for i in range(args.steps)])
                for j, nm in enumerate(names)}

    # end-to-end through the public API with host buffers
    torch.cuda.synchronize()
    barrier()
    e0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + args.steps + i, host=True)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks((time.perf_counter() - e0) * 1e3)

    pk = peaks()
    ms_step = ms / args.steps
    value = PAIRS_PER_STEP * world / (ms_step * 1e-3)
    # dominant kernel by time share among the algorithmic stages
    dom = max(ALG, key=lambda k: stage_ms[k])
    kind, work = ALG[dom]
    alu_ops = N_SMS * FP32_LANES * pk["sm_max_mhz"] * 1e6
    if kind == "alu_flop":
        peak, unit, achieved = 2 * alu_ops / 1e12, "TFLOP/s", work(n) / (stage_ms[dom] * 1e-3) / 1e12
    else:
        peak, unit, achieved = alu_ops / 1e12, "Tops/s", work(n) / (stage_ms[dom] * 1e-3) / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if os.path.exists(tpath):
        traffic = json.load(open(tpath)).get(CFG["name"], {}).get(dom)
    rp, rs, rk, rh = res
    if args.workload != "focus":
        rk = rh = [{"max": None}]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "point-pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded Gaussian random field + latent signal; stand-in for the "
                "paper's ensembles)",
        "config": {"workload": CFG["name"] if args.workload == "focus" else
                   CFG["name"] + "-regions-only",
                   "field": "352x256x20" if args.workload == "focus" else "two 32x32x20 boxes",
                   "members": n,
                   "regions": "2 x 32x32x20 (20480 points each)",
                   "allpairs_per_measure": N_ALL, "sampled_pairs": N_SAMPLED,
                   "ksg_k": CFG["k"], "hist_bins": CFG["bins"],
                   "l2": "inputs larger than L2 (field 721 MB rewritten as 4.6 GB of planes "
                         "every step)",
                   "parallelism": f"replicas x{world}"},
        "measures": {
            "pearson_allpairs_pairs_per_s": N_ALL / (stage_ms["allpairs_pearson"] * 1e-3),
            "spearman_allpairs_pairs_per_s": N_ALL / (stage_ms["allpairs_spearman"] * 1e-3),
            "ksg_pairs_per_s": N_SAMPLED / (stage_ms["ksg"] * 1e-3),
            "hist_pairs_per_s": N_SAMPLED / (stage_ms["hist"] * 1e-3),
            "stage_ms": stage_ms,
        },
        "results": {"pearson_max": rp["max"], "spearman_max": rs["max"], "ksg_max": rk[0]["max"],
                    "hist_max": rh[0]["max"]},
        "roofline": {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": unit, "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"derived: {N_SMS} SMs x {FP32_LANES} FP32 lanes x "
                                    f"{pk['sm_max_mhz']:.0f} MHz (MEASURED_PEAKS sm_max_mhz)"},
        "e2e": {"value": PAIRS_PER_STEP * world / (e2e_ms / args.steps * 1e-3),
                "unit": "point-pairs/s",
                "h2d_bytes_per_step": int(F_host.nbytes),
                "d2h_bytes_per_step": int(2 * 4 * N_SAMPLED + 4 * 40)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    cc.close()
    return line


# ----------------------------------------------------------------------------- oracle
def oracle_sample_rates(F, threads=None, budget_s=12.0):
    """Time the FP64 oracle on bounded samples of each stage; seconds per pair."""
    import oracle
    o = oracle.get()
    if threads:
        o.set_threads(threads)
    A = oracle.box_points(CFG["X"], CFG["Y"], CFG["Z"], CFG["box_a"])
    B = oracle.box_points(CFG["X"], CFG["Y"], CFG["Z"], CFG["box_b"])
    rng = np.random.default_rng(99)
    rates = {}
    plan = [("allpairs_pearson", oracle.PEARSON, {}, 40000),
            ("allpairs_spearman", oracle.SPEARMAN, {}, 20000),
            ("ksg", oracle.MI_KSG, {"k": CFG["k"]}, 4000),
            ("hist", oracle.MI_BINNED, {"bins": CFG["bins"]}, 40000)]
    per = budget_s / len(plan)
    samples = {}
    for name, kind, kw, m in plan:
        ia = A[rng.integers(0, len(A), m)]
        ib = B[rng.integers(0, len(B), m)]
        t = time.perf_counter()
        o.eval_pairs(F, kind, ia[:64], ib[:64], **kw)
        t64 = (time.perf_counter() - t) / 64
        m = int(max(64, min(m, per / max(t64, 1e-9))))
        t = time.perf_counter()
        o.eval_pairs(F, kind, ia[:m], ib[:m], **kw)
        rates[name] = (time.perf_counter() - t) / m
        samples[name] = m
    return rates, samples, o.threads()


def oracle_step_seconds(rates):
    return (rates["allpairs_pearson"] * N_ALL + rates["allpairs_spearman"] * N_ALL +
            (rates["ksg"] + rates["hist"]) * N_SAMPLED)


def cpu_baseline_line(F):
    rates, samples, cores = oracle_sample_rates(F)
    t = oracle_step_seconds(rates)
    return {"value": PAIRS_PER_STEP / t, "unit": "point-pairs/s", "cores": cores, "kind": "oracle",
            "sample": "FP64 oracle timed on " + ", ".join(f"{v} {k} pairs" for k, v in
                                                         samples.items()) +
                      " drawn from the step's region pair; per-pair time scaled to the step"}


def run_reference(args):
    F = gen.field(CFG["seed"], CFG["X"], CFG["Y"], CFG["Z"], CFG["n"])
    import oracle
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample_rates(F, budget_s=budget)
    times, samples, cores = [], None, None
    for _ in range(args.steps):
        rates, samples, cores = oracle_sample_rates(F, budget_s=budget)
        times.append(oracle_step_seconds(rates))
    t = statistics.median(times)
    value = PAIRS_PER_STEP / t
    desc = ("FP64 oracle on " + ", ".join(f"{v} {k} pairs" for k, v in samples.items()) +
            " per step, scaled to the full step")
    return {"metric": METRIC, "value": value, "unit": "point-pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": CFG["name"], "members": CFG["n"]},
            "cpu_baseline": {"value": value, "unit": "point-pairs/s", "cores": cores,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "point-pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="focus", choices=["focus", "focus-regions"],
                    help="focus-regions generates only the two boxes (small case for ncu)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu_baseline:
            F = gen.field(CFG["seed"], CFG["X"], CFG["Y"], CFG["Z"], CFG["n"])
            line["cpu_baseline"] = cpu_baseline_line(F)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
