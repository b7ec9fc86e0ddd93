#!/usr/bin/env python3
"""Benchmark: contracted SHG two-center integrals on GB300.

One step = every two-center block of the 2,000,000-pair high-l workload
(la, lb in 0..6 with P(l) ~ 2^-l, contraction lengths 1..20 with 30% of the
shells at 12..20 primitives, exponents 0.03..5000, separations 0..10 bohr,
seed 2) for 1/r and erfc(0.11 r)/r, i.e. 4,000,000 shell-pair integrals:
one fused persistent launch for both operators in FP64 (--precision mixed:
double-float; --separate: one persistent launch per operator).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp64|mixed] [--separate] [--configs]

N > 1 runs under torch.distributed.run, one rank per GPU: the one pair list
is split into cost-balanced contiguous slices, one per rank (shard.py; strong
scaling, no data-path collective: each rank writes its own blocks), and the
step time is the maximum over the ranks (--replicas: every rank evaluates the
whole workload, weak scaling).  Prints one JSON line on rank 0.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shell-pair integrals/s on 1 GB300 at 1e-12 rel (FP64) vs mixed; % of roofline"
UNIT = "shell-pair integrals/s"
WORKLOAD = "c3_2m_l6_k20"
OPS = [("coulomb", 1, 0.0), ("erfc", 2, 0.11)]
DF_FMA_FP32_INSTR = 18.0       # FP32 instructions of one double-float multiply-add
FP64_NOMINAL_TFLOPS = 1.25   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal, context)
PROFILES = {"fp64_fused": os.path.join(ROOT, "profiles", "k_2c_fp64_fused_persistent_c3_2m.txt"),
            "mixed_fused": os.path.join(ROOT, "profiles", "k_2c_mixed_fused_persistent_c3_2m.txt"),
            "fp64": os.path.join(ROOT, "profiles", "k_2c_fp64_persistent_c3_2m.txt"),
            "mixed": os.path.join(ROOT, "profiles", "k_2c_mixed_persistent_c3_2m.txt")}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--replicas", action="store_true",
                   help="N > 1: every rank evaluates the whole workload (weak scaling) instead of its "
                        "cost-balanced slice of the one pair list (strong scaling, the default)")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--e2e-chunks", type=int, default=0,
                   help="contiguous chunks of the end-to-end pipeline (read-back of chunk k overlaps chunk k+1); "
                        "0: the pipeline's default for the precision")
    p.add_argument("--n-pairs", type=int, default=None, help="smaller case of the same recipe (profiling only)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                   help="precision of the headline path (the other forms are reported beside it)")
    p.add_argument("--separate", action="store_true",
                   help="headline as one pass per operator instead of the fused multi-operator pass")
    p.add_argument("--no-extras", action="store_true", help="time only the headline path (profiling)")
    p.add_argument("--no-tune", action="store_true", help="default launch shape instead of the autotuner (profiling)")
    p.add_argument("--profile-case", default=None, choices=["aab", "aab_grad", "grad", "family"],
                   help="run one kernel of another workload at size --case-n (profiling captures only)")
    p.add_argument("--case-n", type=int, default=None)
    p.add_argument("--configs", action="store_true",
                   help="also time the other workloads (2k, 2M high-l, (aab) 20k atom pairs, gradients) and add "
                        "them under other_configs")
    return p.parse_args()


def workload_description(n):
    return ("%s: %d shell pairs (la, lb in 0..6 with P(l) ~ 2^-l, contraction lengths 1..11 for 70%% of the "
            "shells and 12..20 for 30%%, exponents log-uniform 0.03..5000, coefficients uniform -1..1 "
            "shell-normalised, separation uniform 0..10 bohr, seed 2) x 2 operators (1/r, erfc(0.11r)/r)"
            % (WORKLOAD, n))


# --------------------------------------------------------------------------- #
# clocks                                                                      #
# --------------------------------------------------------------------------- #
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- #
# CPU oracle baseline                                                         #
# --------------------------------------------------------------------------- #
def oracle_stratified(shells, pa, pb, budget_s, nthreads, seed=11):
    """Oracle throughput on the workload, estimated from a class-stratified sample.

    Every (la, lb) class of the pair list is timed on its own random sample
    (the contraction lengths inside a class in their workload proportions),
    n_c pairs of the class's N_c, all operators; the workload's time is
    extrapolated as sum_c (N_c / n_c) T_c.  The sample is sized from a pilot
    so that it takes about budget_s, with at least min(N_c, 16) pairs per
    class.  Runs the FP64 build of the oracle on nthreads OpenMP threads."""
    import numpy as np
    import oracle
    from paper_1701_06588_gb300 import workloads as W
    l = np.asarray(shells["l"])
    cls = l[pa] * 7 + l[pb]
    rng = np.random.default_rng(seed)

    def run(idx):
        sub, spa, spb = W.subset_pairs(shells, pa, pb, np.sort(idx))
        t0 = time.perf_counter()
        for _, op, om in OPS:
            oracle.eval_2c(sub, spa, spb, op, om, nthreads=nthreads, long_double=False)
        return time.perf_counter() - t0

    pilot = rng.choice(len(pa), min(len(pa), 256), replace=False)
    run(pilot[:16])
    per_pair = run(pilot) / len(pilot)
    frac = min(1.0, budget_s / max(per_pair * len(pa), 1e-9))
    t_est, n_sample, t_sample = 0.0, 0, 0.0
    for c in np.unique(cls):
        members = np.where(cls == c)[0]
        n_c = int(min(len(members), max(min(len(members), 16), round(frac * len(members)))))
        t_c = run(rng.choice(members, n_c, replace=False))
        t_est += len(members) / n_c * t_c
        n_sample += n_c
        t_sample += t_c
    rate = len(pa) * len(OPS) / t_est
    sample = ("class-stratified sample of %s: %d of %d pairs over %d (la, lb) classes (contraction lengths in "
              "their workload proportions inside each class) x %d operators, %.1f s of oracle time; throughput "
              "extrapolated to the whole workload as sum_c N_c/n_c T_c; FP64 build of the Obara-Saika oracle, "
              "%d OpenMP threads (a reported baseline, not a tuned competitor)"
              % (WORKLOAD, n_sample, len(pa), len(np.unique(cls)), len(OPS), t_sample, nthreads))
    return rate, t_sample, sample


def cpu_baseline(shells, pa, pb, budget_s=20.0):
    nthreads = os.cpu_count() or 1
    rate, _, sample = oracle_stratified(shells, pa, pb, budget_s, nthreads)
    return {"value": rate, "unit": UNIT, "cores": nthreads, "kind": "oracle", "sample": sample}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, on the host cores; every
    step is a class-stratified sample of the workload (see oracle_stratified)."""
    from paper_1701_06588_gb300 import workloads as W
    if rank != 0:
        return
    shells, pa, pb = W.make(WORKLOAD)
    nthreads = os.cpu_count() or 1
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_stratified(shells, pa, pb, budget / 4, nthreads)
    rates, times = [], []
    sample = ""
    for s in range(args.steps):
        r, t, sample = oracle_stratified(shells, pa, pb, budget, nthreads, seed=100 + s)
        rates.append(r)
        times.append(t)
    value = statistics.mean(rates)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * len(pa) * len(OPS) / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_description(len(pa)), "sample": sample,
                   "ms_per_step": "extrapolated time of one whole step; each step timed %.1f s of oracle work on "
                                  "its sample" % statistics.mean(times)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# --------------------------------------------------------------------------- #
# GPU arm                                                                     #
# --------------------------------------------------------------------------- #
# the sources that build the two-center kernels the profiles describe (their
# device code, tables and launch logic); the (aab), family, gradient and
# allocation-free translation units are not part of them
KERNEL_SOURCES = ["shg_api.cpp", "shg_device.cuh", "shg_df.cuh", "shg_fused.cu", "shg_grad_angular.cuh",
                  "shg_internal.h", "shg_kernels.cu", "shg_mix_angular.cuh", "shg_mixed.cu"]


def kernel_sources_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1701_06588_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def read_profile_traffic(precision):
    """DRAM bytes per step of the timed kernels from the committed ncu summary,
    or None when it is absent or was taken on other kernel sources."""
    try:
        kv = {}
        for ln in open(PROFILES[precision]):
            if ":" in ln:
                k, v = ln.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_sources_sha") != kernel_sources_sha():
            return None
        return float(kv["dram_bytes_per_step"])
    except Exception:
        return None


def rank_workload(shells, pa, pb, rank, world, replicas=False):
    """The pairs this rank evaluates.  One rank, or replicas: the whole list.
    Otherwise the cost-balanced contiguous slice of the one list that
    shard.shard_bounds gives rank `rank` of `world` (estimated FP64 flops of
    the count model), with its shells only.  Returns (shells, pair_a, pair_b,
    first pair index, units of the whole job per step)."""
    from paper_1701_06588_gb300 import shard, workloads as W
    if world == 1 or replicas:
        return shells, pa, pb, 0, world * len(pa) * len(OPS)
    b = shard.shard_bounds(shard.pair_costs(shells["l"], shells["nprim"], pa, pb), world)
    lo, hi = int(b[rank]), int(b[rank + 1])
    sub, spa, spb = W.subset_pairs(shells, pa, pb, range(lo, hi))
    return sub, spa, spb, lo, len(pa) * len(OPS)


def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_1701_06588_gb300 import api, autotune, build, counts, workloads as W
    from paper_1701_06588_gb300 import _lib as L

    build.build()
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    shells, pa, pb = W.make(WORKLOAD, n=args.n_pairs)
    n_pairs_job = len(pa)
    shells, pa, pb, first_pair, job_units = rank_workload(shells, pa, pb, rank, world, args.replicas)
    n_pairs = len(pa)
    units_per_step = n_pairs * len(OPS)
    basis = api.Basis(shells)
    off, total = basis.pair_offsets(pa, pb)
    d_off = torch.from_numpy(off).cuda()
    outs = [torch.empty(total, dtype=torch.float64, device="cuda") for _ in OPS]
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    s_handle = stream.cuda_stream
    names = [o[0] for o in OPS]
    omegas = [o[2] for o in OPS]

    fp64_peak = max(L.shg_measure_alu_peak(0, 4096, s_handle) for _ in range(3))
    fp32_peak = max(L.shg_measure_alu_peak(1, 65536, s_handle) for _ in range(2))
    dmma_peak = max(L.shg_measure_alu_peak(2, 1024, s_handle) for _ in range(2))

    def time_steps(step_fn, steps, per_op=False):
        """K steps, L2 flushed between steps outside the events; per-step ms
        (and per-operator ms when per_op)."""
        ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in (OPS if per_op else [0])] for _ in range(steps)]
        for s in range(steps):
            flush.zero_()
            step_fn(ev[s])
        torch.cuda.synchronize()
        if per_op:
            per = [statistics.mean(ev[s][i][0].elapsed_time(ev[s][i][1]) for s in range(steps)) for i in range(len(OPS))]
            return sum(per), per
        return statistics.mean(ev[s][0][0].elapsed_time(ev[s][0][1]) for s in range(steps)), None

    def plan_step(plan, precision):
        def fn(evs):
            for (name, _, om), o, (e0, e1) in zip(OPS, outs, evs):
                e0.record(stream)
                plan.exec(name, d_off, o, omega=om, precision=precision)
                e1.record(stream)
        return fn

    def fused_step(plan):
        def fn(evs):
            e0, e1 = evs[0]
            e0.record(stream)
            plan.exec_fused(names, d_off, outs, omegas=omegas, precision=args.precision)
            e1.record(stream)
        return fn

    def graph_step(graph):
        def fn(evs):
            e0, e1 = evs[0]
            e0.record(stream)
            graph.launch()
            e1.record(stream)
        return fn

    # headline form: the fused multi-operator pass (one kernel per step) unless --separate
    fused = not args.separate
    form = args.precision + ("_fused" if fused else "")
    # autotuned launch shape for each form (cached per GPU and workload)
    tuned = {}
    for f in ("fp64_fused", "fp64", "mixed_fused", "mixed"):
        if args.no_extras and f != form:
            continue
        if args.no_tune:
            tuned[f] = {"schedule": "persistent", "threads_per_cta": 128, "ctas_per_sm": 0, "variant": 1}
        else:
            tuned[f] = autotune.tune_2c(basis, pa, pb, names, omegas, d_off, outs, precision=f)

    # headline: the autotuned plan of the headline form, replayed as one CUDA graph per step
    plan = autotune.tuned_plan(basis, pa, pb, tuned[form])
    graph = api.Graph2c(plan, names, omegas, d_off, outs, precision=args.precision, fused=fused)
    kern_step = fused_step(plan) if fused else plan_step(plan, args.precision)
    for _ in range(max(args.warmup, 0)):
        graph.launch()
        kern_step([(torch.cuda.Event(enable_timing=True),) * 2 for _ in OPS])
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ms_step, _ = time_steps(graph_step(graph), args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    # kernel time of the same plan (same kernels, launched outside the graph; per operator
    # for the separate passes)
    kern_ms, per_op_ms = time_steps(kern_step, args.steps, per_op=not fused)
    if dist:
        t = torch.tensor([ms_step], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = job_units / (ms_step * 1e-3)

    flops_separate = sum(counts.workload_flops(shells, pa, pb, op) for _, op, _ in OPS)
    # the fused passes sum the far field of 1/r (T >= 120) as one multiply-add per
    # primitive pair: count those pairs exactly
    n_far = counts.far_primitive_pairs(shells, pa, pb) if fused else None
    flops_step = (counts.workload_fused_flops(shells, pa, pb, [(op, om) for _, op, om in OPS], n_far) if fused
                  else flops_separate)
    achieved = flops_step / (kern_ms * 1e-3) / 1e12
    # double-float: one multiply-add of the FP64 formula costs 18 FP32 instructions
    # (TwoProd 4, FastTwoSum 3, TwoSum 6, 2 adds, FastTwoSum 3), so the FP32 FMA rate
    # (2 flops per instruction) bounds FP64-formula flops at fp32_peak / 18
    peak = (fp64_peak if args.precision == "fp64" else fp32_peak / DF_FMA_FP32_INSTR) / 1e12
    traffic = read_profile_traffic(form)

    forms = {}
    if not args.no_extras:
        # plain per-class FP64 (the baseline the mixed, autotuned, graph form is compared with)
        pc = api.Plan2c(basis, pa, pb, schedule="per_class")
        plan_step(pc, "fp64")([(torch.cuda.Event(enable_timing=True),) * 2 for _ in OPS])
        ms_pc, _ = time_steps(plan_step(pc, "fp64"), args.steps, per_op=True)
        forms["fp64_per_class"] = {"ms_per_step": ms_pc, "value": units_per_step / (ms_pc * 1e-3),
                                   "launches_per_step": len(OPS) * pc.launches}
        pc.close()
        pp = api.Plan2c(basis, pa, pb, schedule="persistent")
        ms_pp, _ = time_steps(plan_step(pp, "fp64"), args.steps, per_op=True)
        forms["fp64_persistent"] = {"ms_per_step": ms_pp, "value": units_per_step / (ms_pp * 1e-3)}
        pp.close()
        for other in ("fp64_fused", "fp64", "mixed_fused", "mixed"):
            if other == form:
                continue
            po = autotune.tuned_plan(basis, pa, pb, tuned[other])
            go = api.Graph2c(po, names, omegas, d_off, outs, precision="mixed" if other.startswith("mixed") else "fp64",
                             fused=other.endswith("_fused"))
            go.launch()
            torch.cuda.synchronize()
            ms_o, _ = time_steps(graph_step(go), args.steps)
            forms[other + "_tuned_graph"] = {"ms_per_step": ms_o, "value": units_per_step / (ms_o * 1e-3),
                                             "launch": {k: tuned[other].get(k, 0) for k in
                                                        ("schedule", "threads_per_cta", "ctas_per_sm", "variant")}}
            go.close()
            po.close()
        forms[form + "_tuned_graph"] = {"ms_per_step": ms_step, "value": units_per_step / (ms_step * 1e-3),
                                        "launch": {k: tuned[form].get(k, 0) for k in
                                                   ("schedule", "threads_per_cta", "ctas_per_sm", "variant")}}
        for f in ("fp64_fused", "mixed_fused", "mixed"):
            forms[f + "_speedup_vs_fp64_per_class"] = ms_pc / forms[f + "_tuned_graph"]["ms_per_step"]
            forms[f + "_speedup_vs_fp64_tuned_graph"] = (forms["fp64_tuned_graph"]["ms_per_step"] /
                                                         forms[f + "_tuned_graph"]["ms_per_step"])
        torch.cuda.synchronize()

    # end to end through the public API with host buffers
    cent_h = torch.from_numpy(np.ascontiguousarray(shells["centers"])).pin_memory()
    pa_h = torch.from_numpy(pa).pin_memory()
    pb_h = torch.from_numpy(pb).pin_memory()
    off_h = torch.from_numpy(off).pin_memory()
    outs_h = [torch.empty(total, dtype=torch.float64, pin_memory=True) for _ in OPS]
    d_pa = torch.empty_like(pa_h, device="cuda")
    d_pb = torch.empty_like(pb_h, device="cuda")
    d_off2 = torch.empty_like(off_h, device="cuda")
    copy_stream = torch.cuda.Stream()
    copy_streams = [torch.cuda.Stream() for _ in OPS]
    e2e_times = []
    parts = {"h2d_and_set_centers": [], "plan_create": [], "exec_and_d2h": []}
    for it in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        d_pa.copy_(pa_h, non_blocking=True)
        d_pb.copy_(pb_h, non_blocking=True)
        d_off2.copy_(off_h, non_blocking=True)
        basis.set_centers(cent_h.numpy())
        t2 = time.perf_counter()
        p2 = autotune.tuned_plan(basis, d_pa, d_pb, tuned[form])
        t3 = time.perf_counter()
        if fused:
            p2.exec_fused(names, d_off2, outs, omegas=omegas, precision=args.precision)
            # the outputs read back concurrently, one copy stream each
            done = torch.cuda.Event()
            done.record()
            for o, oh, cs in zip(outs, outs_h, copy_streams):
                cs.wait_event(done)
                with torch.cuda.stream(cs):
                    oh.copy_(o, non_blocking=True)
        for (name, _, om), o, oh in ([] if fused else zip(OPS, outs, outs_h)):
            p2.exec(name, d_off2, o, omega=om, precision=args.precision)
            # read each operator's blocks back on a copy stream while the next operator computes
            done = torch.cuda.Event()
            done.record()
            copy_stream.wait_event(done)
            with torch.cuda.stream(copy_stream):
                oh.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        p2.close()
        if it > 0:
            e2e_times.append(t4 - t1)
            parts["h2d_and_set_centers"].append(t2 - t1)
            parts["plan_create"].append(t3 - t2)
            parts["exec_and_d2h"].append(t4 - t3)
    e2e_single_s = statistics.mean(e2e_times) if e2e_times else float("nan")
    e2e_s = e2e_single_s
    e2e_chunks = args.e2e_chunks or api.HostPipeline2c.default_chunks(args.precision)
    if fused:
        # the public pipeline: the pair list planned in contiguous chunks, each
        # chunk's read-back overlapping the next chunk's fused pass
        pipe = api.HostPipeline2c(basis, n_chunks=e2e_chunks, launch=tuned[form])
        times = []
        for it in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            pipe.run(pa_h, pb_h, off_h, names, outs_h, omegas=omegas, precision=args.precision,
                     centers=cent_h.numpy())
            torch.cuda.synchronize()
            if it > 0:
                times.append(time.perf_counter() - t1)
        if times:
            # median: a host-timed call with 128 MB in and 268 MB out through the
            # host link is exposed to outliers (other traffic on the link)
            e2e_s = statistics.median(times)
    if dist:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = cent_h.numel() * 8 + pa_h.numel() * 4 + pb_h.numel() * 4 + off_h.numel() * 8
    d2h = sum(o.numel() * 8 for o in outs_h)

    dtype = "f64" if args.precision == "fp64" else "f32x2 (double-float) with f64 output"
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak" if (world == 1 or args.replicas) else "strong", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic",
        "config": {"workload": workload_description(n_pairs_job), "pairs": n_pairs_job, "operators": names,
                   "parallelism": ("1 GPU" if world == 1 else
                                   "%d replicas of the whole workload" % world if args.replicas else
                                   "dp%d: cost-balanced contiguous slices of the one pair list (shard.py), no "
                                   "data-path collective; rank 0 evaluates pairs [%d, %d)" %
                                   (world, first_pair, first_pair + n_pairs)),
                   "precision": args.precision,
                   "form": ("fused multi-operator pass (one kernel per step, geometry-only Q_j shared by the "
                            "operators), autotuned launch shape, one CUDA graph per step" if fused else
                            "one pass per operator, autotuned launch shape, one CUDA graph per step"),
                   "launch": {k: tuned[form].get(k, 0) for k in ("schedule", "threads_per_cta", "ctas_per_sm", "variant")},
                   "units_per_step": job_units, "units_per_step_this_rank": units_per_step,
                   "elements_per_step_this_rank": total * len(OPS),
                   "l2": "flushed between steps by a 512 MB device write outside the timed events",
                   "wall_s_timed_loop": wall},
        "per_operator_kernel_ms": {n: m for n, m in zip(names, per_op_ms)} if per_op_ms else None,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "peak_source": ("measured FP64 FMA-chain probe (shg_measure_alu_peak) in this run; nominal %.2f "
                                     "TFLOP/s = 152 SMs x 2 FMA/clk x 2 x 2.07 GHz" % FP64_NOMINAL_TFLOPS)
                     if args.precision == "fp64" else
                     "double-float rate derived from the measured FP32 FMA-chain probe (shg_measure_alu_peak) "
                     "in this run: FP32 rate / 18 (FP32 instructions of one double-float multiply-add); "
                     "algorithmic flops are the FP64 formula count",
                     "algorithmic_flops_per_step": flops_step, "kernel_ms_per_step": kern_ms,
                     "far_field_primitive_pairs": (int(n_far.sum()) if n_far is not None else None),
                     "separate_passes_flops_per_step": flops_separate,
                     "kernel": ("k_2c_%s_fused_persistent (1/r and erfc in one pass)" %
                                ("fp64" if args.precision == "fp64" else "mixed") if fused else
                                "k_2c_%s_persistent<op> / static (one launch per operator)" %
                                ("fp64" if args.precision == "fp64" else "mixed"))},
        "forms": forms,
        "e2e": {"value": job_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "what": ("per step, api.HostPipeline2c: shg_basis_set_centers from pinned host centers, then the "
                         "pair list in %d contiguous chunks; per chunk the pinned H2D of its pair lists and "
                         "offsets and shg_plan_2c_create on an upload stream (overlapping the previous chunk's "
                         "pass), shg_plan_2c_exec_fused (both operators), and the D2H of its blocks to pinned "
                         "memory on a copy stream overlapping the next chunk; median over the timed calls"
                         % e2e_chunks if fused else
                         "per step: pinned H2D of pair lists, offsets and centers, shg_basis_set_centers, "
                         "shg_plan_2c_create, one shg_plan_2c_exec per operator, D2H of all blocks to pinned memory (operator "
                         "k's copy on a second stream overlaps operator k+1's kernel)"),
                "unchunked_ms": 1e3 * e2e_single_s,
                "unchunked_ms_parts": {k: 1e3 * statistics.mean(v) for k, v in parts.items() if v}},
        "gpu_launches": args.steps * (1 if fused else len(OPS)) * plan.launches_for(args.precision),
        "clocks": clk,
        "measured_peaks_tflops": {"fp64": fp64_peak / 1e12, "fp32": fp32_peak / 1e12,
                                  "fp64_tensor_mma_m8n8k4": dmma_peak / 1e12},
    }
    if args.configs:
        result["other_configs"] = other_configs(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(shells, pa, pb)
    if rank == 0:
        print(json.dumps(result), flush=True)
    graph.close()
    plan.close()
    basis.close()
    if dist:
        dist.destroy_process_group()


def _events_ms(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def profile_case(args):
    """One warm and one timed call of a single kernel at a moderate size, for
    ncu captures of the kernels outside the headline step:
      aab       (a b a~) FP64, n atom pairs of the 20,000-atom-pair recipe (150 triples each)
      aab_grad  its vector-Jacobian product
      grad      two-center Coulomb VJP, n pairs of the 500k-pair gradient recipe
      family    family-path Coulomb blocks of an n-atom molecule
    Prints one JSON line with the CUDA-event time of the timed call."""
    import numpy as np
    import torch
    from paper_1701_06588_gb300 import _lib as L, api, build, molecule, workloads as W
    build.build()
    st = torch.cuda.current_stream().cuda_stream
    case, n = args.profile_case, args.case_n
    if case in ("aab", "aab_grad"):
        sh, ta, tt, tb, _ = W.make("c4_aab_20k", n=n or 2000)
        b = api.Basis(sh)
        off, total = b.triple_offsets(b, ta, tt, tb)
        d_off = torch.from_numpy(off).cuda()
        d = [torch.from_numpy(x).cuda() for x in (ta, tt, tb)]
        if case == "aab":
            out = torch.empty(total, dtype=torch.float64, device="cuda")
            fn = lambda: L.shg_eval_3c_aab(b.handle, b.handle, len(ta), *d, 0, 0.0, d_off, out, st)
        else:
            w = torch.empty(total, dtype=torch.float64, device="cuda").uniform_(-1, 1)
            ga = torch.empty((len(ta), 3), dtype=torch.float64, device="cuda")
            gb = torch.empty_like(ga)
            fn = lambda: L.shg_eval_3c_aab_grad(b.handle, b.handle, len(ta), *d, 0, d_off, w, ga, gb, st)
        units = len(ta)
    elif case == "grad":
        sh, pa, pb = W.make("c5_grad_500k_l5_k12", n=n or 100_000)
        b = api.Basis(sh)
        off, total = b.pair_offsets(pa, pb)
        d_off, d_pa, d_pb = (torch.from_numpy(x).cuda() for x in (off, pa, pb))
        w = torch.empty(total, dtype=torch.float64, device="cuda").uniform_(-1, 1)
        ga = torch.empty((len(pa), 3), dtype=torch.float64, device="cuda")
        gb = torch.empty_like(ga)
        fn = lambda: L.shg_eval_2c_grad(b.handle, len(pa), d_pa, d_pb, 1, 0.0, 0, d_off, w, ga, gb, st)
        units = len(pa)
    else:
        coords, el, bs = W.molecule_workload(n or 300, seed=7)
        mol = molecule.Molecule(coords, el, bs)
        pa, pb = mol.shell_pairs(True)
        off, total = mol.basis.pair_offsets(pa, pb)
        d_off = torch.from_numpy(off).cuda()
        out = torch.empty(total, dtype=torch.float64, device="cuda")
        fp = api.FamilyPlan(mol.basis, pa, pb)
        fn = lambda: fp.exec("coulomb", d_off, out)
        units = len(pa)
    ms = _events_ms(fn, 1)
    print(json.dumps({"profile_case": case, "units": units, "ms": ms}))


def _plan_create_ms(basis, plan, reps=20):
    """Median host wall time of shg_plan_2c_create + shg_plan_destroy on
    device-resident pair lists (the planner's one synchronisation included)."""
    import torch
    from paper_1701_06588_gb300 import _lib as L
    st = torch.cuda.current_stream().cuda_stream
    ts = []
    for _ in range(reps + 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = L.shg_plan_2c_create(basis.handle, plan.n, plan.pair_a, plan.pair_b, L.SHG_SCHED_PERSISTENT, st)
        L.shg_plan_destroy(h)
        ts.append((time.perf_counter() - t0) * 1e3)
    return sorted(ts[2:])[reps // 2]


def other_configs(args):
    """Throughput of the other synthetic workloads (CUDA events, inputs resident)."""
    import numpy as np
    import torch
    from paper_1701_06588_gb300 import api, workloads as W
    from paper_1701_06588_gb300 import counts
    res = {}
    for key, name, ops, precs in [
            ("c1_2k_l3_k4", "c1_2k_l3_k4", [("overlap", 0.0), ("coulomb", 0.0)], ("fp64", "mixed")),
            ("c2_200k_l4_k8", "c2_200k_l4_k8", [("overlap", 0.0), ("coulomb", 0.0), ("erfc", 0.11), ("erf", 0.11),
                                                ("gauss", 1.0)], ("fp64", "mixed")),
            ("c2_200k_l4_k8 exp(-0.3 r^2)/r", "c2_200k_l4_k8", [("gauss_coulomb", 0.3)], ("fp64", "mixed")),
            ("c2_200k_l4_k8 r_a^4 (n = 2)", "c2_200k_l4_k8", [("ra2n", 2.0)], ("fp64",))]:
        sh, pa, pb = W.make(name)
        b = api.Basis(sh)
        off, total = b.pair_offsets(pa, pb)
        d_off = torch.from_numpy(off).cuda()
        out = torch.empty(total, dtype=torch.float64, device="cuda")
        plan = api.Plan2c(b, pa, pb)
        entry = {"pairs": len(pa), "operators": [o[0] for o in ops], "plan_create_ms": _plan_create_ms(b, plan)}
        flops = sum(counts.workload_flops(sh, pa, pb, api.L.OPERATORS[n]) for n, _ in ops)
        for prec in precs:
            ms = sum(_events_ms(lambda n=n, w=w: plan.exec(n, d_off, out, omega=w, precision=prec), 3 if len(pa) > 1e5
                                else 50) for n, w in ops)
            entry[prec] = {"ms_per_pass": ms, "shell_pair_integrals_per_s": len(pa) * len(ops) / (ms * 1e-3),
                           "algorithmic_tflops": flops / (ms * 1e-3) / 1e12}
        if len(ops) > 1:
            # the same operators in one fused pass
            outs = [out] + [torch.empty(total, dtype=torch.float64, device="cuda") for _ in ops[1:]]
            names, oms = [n for n, _ in ops], [w for _, w in ops]
            ff = counts.workload_fused_flops(sh, pa, pb, [(api.L.OPERATORS[n], w) for n, w in ops],
                                             counts.far_primitive_pairs(sh, pa, pb))
            for prec in precs:
                ms = _events_ms(lambda: plan.exec_fused(names, d_off, outs, omegas=oms, precision=prec),
                                3 if len(pa) > 1e5 else 50)
                entry[prec + "_fused"] = {"ms_per_pass": ms,
                                          "shell_pair_integrals_per_s": len(pa) * len(ops) / (ms * 1e-3),
                                          "algorithmic_tflops": ff / (ms * 1e-3) / 1e12}
            del outs
        res[key] = entry
        plan.close()
        b.close()
        del out
    # (aab): 20,000 atom pairs = 3,000,000 triples
    sh, ta, tt, tb, per = W.make("c4_aab_20k")
    b = api.Basis(sh)
    off, total = b.triple_offsets(b, ta, tt, tb)
    d_off = torch.from_numpy(off).cuda()
    d_ta, d_tt, d_tb = (torch.from_numpy(x).cuda() for x in (ta, tt, tb))
    out = torch.empty(total, dtype=torch.float64, device="cuda")
    from paper_1701_06588_gb300 import _lib as L
    st = torch.cuda.current_stream().cuda_stream
    ms = _events_ms(lambda: L.shg_eval_3c_aab(b.handle, b.handle, len(ta), d_ta, d_tt, d_tb, 0, 0.0, d_off, out, st), 3)
    f3 = counts.workload_triple_flops(sh, ta, tt, tb)
    res["c4_aab_20k"] = {"triples": len(ta), "atom_pairs": len(ta) // per, "fp64": {
        "ms_per_pass": ms, "triples_per_s": len(ta) / (ms * 1e-3), "elements": total,
        "algorithmic_tflops": f3 / (ms * 1e-3) / 1e12}}
    ms = _events_ms(lambda: L.shg_eval_3c_aab(b.handle, b.handle, len(ta), d_ta, d_tt, d_tb, 1, 0.0, d_off, out, st), 3)
    res["c4_aab_20k"]["mixed"] = {"ms_per_pass": ms, "triples_per_s": len(ta) / (ms * 1e-3),
                                  "form": "radial sums FP64, angular part and Gaunt sum double-float"}
    w = torch.empty(total, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    ga = torch.empty((len(ta), 3), dtype=torch.float64, device="cuda")
    gb = torch.empty((len(ta), 3), dtype=torch.float64, device="cuda")
    ms = _events_ms(lambda: L.shg_eval_3c_aab_grad(b.handle, b.handle, len(ta), d_ta, d_tt, d_tb, 0, d_off, w, ga, gb,
                                                   st), 2)
    res["c4_aab_20k"]["grad_fp64"] = {"ms_per_pass": ms, "triples_per_s": len(ta) / (ms * 1e-3)}
    b.close()
    del out, w
    # gradients: 500,000 pairs, Coulomb and erfc(0.11)
    sh, pa, pb = W.make("c5_grad_500k_l5_k12")
    b = api.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    d_off = torch.from_numpy(off).cuda()
    d_pa, d_pb = torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda()
    w = torch.empty(total, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    ga = torch.empty((len(pa), 3), dtype=torch.float64, device="cuda")
    gb = torch.empty((len(pa), 3), dtype=torch.float64, device="cuda")
    entry = {"pairs": len(pa)}
    for opn, op, om in [("coulomb", 1, 0.0), ("erfc", 2, 0.11)]:
        ms = _events_ms(lambda: L.shg_eval_2c_grad(b.handle, len(pa), d_pa, d_pb, op, om, 0, d_off, w, ga, gb, st), 3)
        entry[opn] = {"ms_per_pass": ms, "pair_gradients_per_s": len(pa) / (ms * 1e-3),
                      "algorithmic_tflops": counts.workload_grad_flops(sh, pa, pb, op) / (ms * 1e-3) / 1e12}
        # mixed: double-float radial orders (classes with both l >= 4 in FP64)
        ms = _events_ms(lambda: L.shg_eval_2c_grad(b.handle, len(pa), d_pa, d_pb, op, om, L.SHG_PREC_MIXED, d_off, w,
                                                   ga, gb, st), 3)
        entry[opn + "_mixed"] = {"ms_per_pass": ms, "pair_gradients_per_s": len(pa) / (ms * 1e-3)}
    res["c5_grad_500k_l5_k12"] = entry
    b.close()
    # molecular assembly: 300-atom molecule with family basis sets, all shell pairs a <= b
    from paper_1701_06588_gb300 import molecule
    coords, el, bs = W.molecule_workload(300, seed=7)
    mol = molecule.Molecule(coords, el, bs)
    pa, pb = mol.shell_pairs(True)
    off, total = mol.basis.pair_offsets(pa, pb)
    d_pa, d_pb, d_off = (torch.from_numpy(x).cuda() for x in (pa, pb, off))
    blocks = torch.empty(total, dtype=torch.float64, device="cuda")
    plan = api.Plan2c(mol.basis, d_pa, d_pb)
    M = torch.zeros((mol.nao, mol.nao), dtype=torch.float64, device="cuda")
    ms_eval = _events_ms(lambda: plan.exec("coulomb", d_off, blocks), 5)
    fplan = api.FamilyPlan(mol.basis, d_pa, d_pb)
    ms_fam = _events_ms(lambda: fplan.exec("coulomb", d_off, blocks), 5)
    n_groups = fplan.n_groups
    fplan.close()
    ms_scat = _events_ms(lambda: L.shg_scatter_2c(mol.basis.handle, len(pa), d_pa, d_pb, d_off, blocks,
                                                  mol.d_ao_off, mol.nao, 1, M, st), 5)
    la = mol.shells["l"][pa].astype(np.int64)
    n_el = (2 * la + 1) * (2 * mol.shells["l"][pb].astype(np.int64) + 1)
    offdiag = (pa != pb)
    scat_bytes = float(8 * n_el.sum() + 8 * (n_el * (1 + offdiag)).sum() + 24 * len(pa))
    Wt = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, (mol.nao, mol.nao))).cuda()
    Wt = 0.5 * (Wt + Wt.T)
    ms_mat = _events_ms(lambda: mol.matrix("coulomb"), 3)
    ms_frc = _events_ms(lambda: mol.forces("coulomb", Wt), 3)
    res["molecule_300_atoms"] = {
        "atoms": mol.n_atoms, "shells": len(mol.shells["l"]), "nao": mol.nao, "shell_pairs": len(pa),
        "coulomb_eval_ms": ms_eval, "coulomb_eval_family_path_ms": ms_fam, "family_pair_groups": n_groups,
        "scatter_ms": ms_scat,
        "scatter_gbs": scat_bytes / (ms_scat * 1e-3) / 1e9, "scatter_algorithmic_bytes": scat_bytes,
        "matrix_ms_incl_planning": ms_mat, "forces_ms_incl_planning": ms_frc}
    plan.close()
    mol.close()
    return res


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.profile_case:
        profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
