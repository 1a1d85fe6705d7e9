#!/usr/bin/env python
"""DSRG-MRPT3 energy throughput on GB300.

One step = one full unrelaxed DSRG-MRPT3 energy (first-order amplitudes,
E(2), the second-order transformed Hamiltonian with the density-fitted
particle-particle ladder, rings and cumulant terms, second-order amplitudes,
E(3)) of one synthetic instance, through the library's C interface.

Workload (default): 30 core, CAS(8,8) reference (4900 Ms=0 determinants,
seeded random CI vector with exact gamma1 / lambda2 / lambda3), 300 virtual,
1200 auxiliary functions, s = 0.5 Eh^-2, inputs from the seeded generator in
synth/ (uniform orbital energies per block, symmetric Gaussian B^Q scaled by
0.1 exp(-3Q/naux)).  Headline: the split-precision path (8 digit slices);
the FP64 path is timed on one energy beside it and every energy component
is compared.  The working set (tens of GB) is far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload cas88_c30_v300_q1200|cas66_c10_v100_q400|cas44_c40_v500_q1800|scan32]

Prints one JSON line on rank 0.  With N > 1 (torchrun) every rank computes
its own instance (weak scaling, no collective on the data path).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PT3 energies/sec & effective TFLOP/s: mixed-precision vs FP64 path at ≤1µEh"
WORKLOAD = "cas88_c30_v300_q1200"
# digit slices of the split path per workload: enough for 1e-6 Eh on energies
# of up to 1e4 (6), 1e5 (7) and 1e7 Eh (8)
SLICES = {"cas66_c10_v100_q400": 6, "cas88_c30_v300_q1200": 7, "cas44_c40_v500_q1800": 8, "scan32": 7,
          "cas1616_c10_v100_q400": 6}
# FP64 runs on the SM's FP64 FMA units (no tcgen05 FP64 kind): 152 SMs x
# 2 FP64 FMA per clock per SM x 2 flop x 2.070 GHz maximum SM clock.
FP64_ALU_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def _measured_bf16():
    """bf16 dense peak for a kernel timed inside a long step: the measured
    sustained figure (the burst figure only if no sustained one is given),
    else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        if "bf16_tflops_sustained" in d:
            return float(d["bf16_tflops_sustained"]), "of measured bf16 sustained"
        return float(d["bf16_tflops"]), "of measured bf16 burst"
    return 1700.0, "of fallback bf16 sustained"


MEASURED_BF16, MEASURED_BF16_SOURCE = _measured_bf16()

def profiled_traffic(workload):
    """DRAM bytes per launch of the split-precision tensor-core kernel from
    the committed ncu capture (profiles/k_ozaki_mma_<workload>.md, a line
    'traffic_bytes_per_launch: B' and the SHA-256 of the kernel source the
    counters were taken on).  None when absent or when the source changed."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"k_ozaki_mma_{workload}.md")
    src = os.path.join(ROOT, "paper_1701_02011_gb300", "csrc", "ozaki.cu")
    if not os.path.exists(path):
        return None, None
    rec = {}
    for line in open(path):
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "kernel_source_sha256")):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip().strip("`")
    if "traffic_bytes_per_launch" not in rec:
        return None, None
    if rec.get("kernel_source_sha256") != hashlib.sha256(open(src, "rb").read()).hexdigest():
        return None, f"profiles/k_ozaki_mma_{workload}.md predates the current kernel source"
    return float(rec["traffic_bytes_per_launch"]), f"profiles/k_ozaki_mma_{workload}.md"


# ----------------------------------------------------------------------------
# rank bookkeeping (host logic, testable without a GPU)
# ----------------------------------------------------------------------------

def rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def instance_seed_offset(rank: int) -> int:
    """Each rank gets its own problem of the same sizes (weak scaling)."""
    return 1000 * rank


def aggregate(per_rank_seconds, steps, world):
    """Whole-job throughput: all ranks' energies over the slowest rank's time."""
    t = max(per_rank_seconds)
    return world * steps / t, t


def max_over_ranks(dist, seconds, device="cuda"):
    """The slowest rank's timed region (every rank must call it)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# CPU oracle timing (the baseline, on a bounded sample)
# ----------------------------------------------------------------------------

def cpu_threads():
    """Threads the oracle's numpy/BLAS calls may use on this host."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(k, "").isdigit():
            return int(os.environ[k])
    return os.cpu_count()


class OracleSample:
    """The CPU oracle (oracle.dsrg_df, plain FP64 numpy, as it stands) on a
    bounded part of the benchmark's own instance: its particle-particle
    ladder (Eq. scaling_problem, the dominant O(N^6) step of the energy at
    these sizes), a few spin-orbital output rows at a time, with <pq||rs>
    built from B^Q for those rows.  A whole oracle energy at this size takes
    far longer than a benchmark may run.  The energies/s figure counts the
    ladder alone (every row at the measured time per row) and so is an
    upper bound on the oracle's rate for whole energies."""

    def __init__(self, inst):
        from oracle import dsrg_df
        t0 = time.perf_counter()
        self.s = dsrg_df.LadderSample(inst)
        self.setup_s = time.perf_counter() - t0
        self.next = 0

    def step(self, rows):
        lo = self.next % self.s.nrows
        hi = min(lo + rows, self.s.nrows)
        t0 = time.perf_counter()
        self.s.rows(lo, hi)
        dt = time.perf_counter() - t0
        self.next = hi
        return dt, hi - lo

    def rate(self, seconds, rows):
        return rows / (seconds * self.s.nrows)

    def text(self, rows_done, seconds):
        return (f"oracle.dsrg_df particle-particle ladder of this instance, {rows_done} of its {self.s.nrows} "
                f"spin-orbital output rows in {seconds:.2f} s (first-order amplitudes and eta.eta.T2 formed "
                f"beforehand in {self.setup_s:.1f} s, not counted); energies/s = rows / (time x all rows): the "
                f"ladder alone, an upper bound on the oracle's rate for whole energies")


def _cpu_baseline_main(workload, seconds, queue):
    import synth
    inst = synth.config_instance(workload)
    smp = OracleSample(inst)
    secs, rows = 0.0, 0
    while (secs < seconds or rows == 0) and rows < smp.s.nrows:
        dt, nr = smp.step(1)
        secs += dt
        rows += nr
    queue.put({"value": smp.rate(secs, rows), "unit": "energies/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": smp.text(rows, secs)})


def cpu_baseline_child(workload, seconds):
    """The oracle sample in a spawned child process (this process holds a
    CUDA context), so that a host-memory failure of the sample cannot take
    the GPU measurement with it."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_cpu_baseline_main, args=(workload, seconds, q))
    p.start()
    out = None
    try:
        out = q.get(timeout=1800)
    except Exception as e:  # noqa: BLE001 - the child died or timed out
        out = {"value": None, "unit": "energies/s", "kind": "oracle", "cores": cpu_threads(),
               "sample": f"oracle sample failed: {type(e).__name__} (exit code {p.exitcode})"}
    p.join(timeout=60)
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    import synth
    wl = args.workload if args.workload != "scan32" else WORKLOAD
    inst = synth.config_instance(wl)
    smp = OracleSample(inst)
    for _ in range(args.warmup):
        smp.step(args.ref_rows)
    secs, rows = [], 0
    for _ in range(args.steps):
        dt, nr = smp.step(args.ref_rows)
        secs.append(dt)
        rows += nr
    tot = sum(secs)
    value = smp.rate(tot, rows)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "energies/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(inst, wl),
        "cpu_baseline": {"value": value, "unit": "energies/s", "cores": cpu_threads(), "kind": "oracle",
                         "sample": smp.text(rows, tot)},
        "e2e": {"value": value, "unit": "energies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": "each step evaluates --ref-rows rows of the oracle's ladder; ms_per_step is that sample's time",
    }
    print(json.dumps(line), flush=True)


def config_dict(inst, workload):
    import synth
    na = inst["na"]
    from math import comb
    dets = comb(na, na // 2) ** 2
    ref = (f"synthetic gamma1 / lambda2 / lambda3 of a {na}-orbital active space (symmetries of cumulants, "
           "no CI vector)" if workload in synth.SYNTHETIC_CONFIGS else f"CAS({na},{na}) Ms=0, {dets} determinants")
    return {"workload": workload, "nc": inst["nc"], "na": na, "nv": inst["nv"], "naux": inst["naux"],
            "s": inst["s"], "reference": ref,
            "l2": "inputs and working set larger than L2; L2 also flushed (256 MiB write) before each timed step"}


def input_bytes(inst):
    import numpy as np
    tot = 0
    for k in ("eps", "B", "g1a", "g1b", "l2aa", "l2ab", "l2bb", "l3aaa", "l3aab", "l3abb", "l3bbb"):
        tot += np.asarray(inst[k]).nbytes
    return tot


def alg_flops(inst, steps):
    """Algorithmic flops of one PT3 energy, fixed before measuring:
    F_lad = h (h+1) v^4 (spatial ladder over i <= j), F_build = Q v^2 (v^2+1)
    ((eg|fh) under pair exchange), F_ring = 2 h^3 p^3 k_ring (k_ring = ring
    products of that shape in the energy's term list), F_low = every other
    contraction as counted by the library (2 M N K each).  h = core +
    active, p = active + virtual, v = virtual, Q = auxiliary.  `steps`: the
    library's per-step FP64 flop counts of a profiled energy."""
    h = inst["nc"] + inst["na"]
    p = inst["na"] + inst["nv"]
    v, Q = inst["nv"], inst["naux"]
    f_lad = h * (h + 1) * v ** 4
    f_build = Q * v * v * (v * v + 1)
    unit = 2.0 * h ** 3 * p ** 3
    ring = steps.get("ring", {}).get("flops", 0.0)
    total = sum(x["flops"] for x in steps.values())
    counted_ladder = sum(steps.get(k, {}).get("flops", 0.0) for k in ("ladder-build", "ladder-contract"))
    f_low = total - counted_ladder - ring
    return {"F_lad": f_lad, "F_build": f_build, "F_ring": ring, "k_ring": ring / unit if unit else 0.0,
            "F_low": f_low, "F_alg": f_lad + f_build + ring + f_low,
            "library_counted_total": total, "library_counted_ladder": counted_ladder}


def _time_path(g, torch, dev, stream, flush, steps, warmup, precision, slices, clocks=None, tune=False,
               profile=True):
    """Warm up, then time `steps` PT3 energies (CUDA events on the library's
    stream around each step, L2 flushed before each step), then run one more
    energy with per-kernel events for the kernel breakdown (kept out of the
    timed steps, whose launches it would slow down)."""
    prec = g.DSRG_PREC_SPLIT if precision == "split" else g.DSRG_PREC_FP64
    h = g.Dsrg(dev, stream=stream.cuda_stream, precision=prec, slices=slices if precision == "split" else 0,
               tune=tune and precision == "split")  # tuning happens in the first warm-up energy
    energies = None
    for _ in range(max(warmup, 0)):
        energies = h.pt3()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    launches = 0
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            starts[k].record(stream)
        energies = h.pt3()
        launches += h.launches
        with torch.cuda.stream(stream):
            ends[k].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    stats, step_stats = {}, {}
    if profile:
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        h.profile(True)
        h.pt3()
        torch.cuda.synchronize()
        stats = h.profile_stats()
        step_stats = h.profile_steps()
        h.profile(False)
    return h, ms, energies, stats, step_stats, launches, clk


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_1701_02011_gb300 as g
    import synth
    from paper_1701_02011_gb300 import build as libbuild

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    libbuild.build()
    wl = args.workload
    slices = args.slices or SLICES[wl]
    inst = synth.config_instance(wl, seed=synth.config_seed(wl) + instance_seed_offset(rank))
    stream = torch.cuda.Stream()
    dev = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
           for k, v in inst.items()}
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if dist:
        dist.barrier()
    h, ms, energies, stats, steps, launches, clocks = _time_path(
        g, torch, dev, stream, flush, args.steps, args.warmup, args.precision, slices, ClockSampler(local_rank),
        tune=not args.no_tune)
    if dist:
        dist.barrier()
    total_s = max_over_ranks(dist, sum(ms) / 1000.0)
    value, tmax = aggregate([total_s], args.steps, world)
    ms_per_step = 1000.0 * tmax / args.steps
    peak_bytes = g.dsrg_peak_bytes(h.h)
    # ---- end to end: host buffers (pinned), copies inside the timed region
    host = {}
    for k, v in inst.items():
        if isinstance(v, np.ndarray):
            host[k] = torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()
        else:
            host[k] = v
    e2e_ms = []
    d2h = 0
    for k in range(max(1, min(args.steps, args.e2e_steps))):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.load(host)
        h.pt3()
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
        d2h = g.dsrg_last_d2h_bytes(h.h)
    e2e_value = world * 1000.0 / statistics.median(e2e_ms)
    h.close()
    # ---- the other precision on one energy: speed and per-component accuracy
    other = "fp64" if args.precision == "split" else "split"
    cmp = None
    if not args.no_comparison:
        torch.cuda.empty_cache()
        cw = 1 if wl == "cas66_c10_v100_q400" else 0
        h2, ms2, e_other, _, _, _, _ = _time_path(g, torch, dev, stream, flush, 1, cw, other, slices,
                                                  tune=not args.no_tune, profile=False)
        h2.close()
        diff = {k: energies[k] - e_other[k] for k in ("e2", "e3a", "e3b", "e3")}
        rel = {k: abs(diff[k]) / max(abs(e_other[k]), 1e-300) for k in diff}
        cmp = {"precision": other, "ms_per_step": ms2[0], "value": 1000.0 / ms2[0], "warmup": cw,
               "energies": e_other, "headline_minus_comparison_Eh": diff, "relative": rel,
               "max_abs_Eh": max(abs(x) for x in diff.values()),
               "speedup": ms2[0] / ms_per_step if args.precision == "split" else ms_per_step / ms2[0]}
    # ---- roofline of the dominant kernel (by device time in the profiled energy)
    dom_name, dom = max(stats.items(), key=lambda kv: kv[1]["ms"])
    step_s = total_s / args.steps
    tensor_kernel = dom_name == "k_ozaki_mma"
    peak = MEASURED_BF16 if tensor_kernel else FP64_ALU_PEAK_TFLOPS
    sec = dom["ms"] / 1000.0
    achieved = dom["flops"] / sec / 1e12 if sec > 0 else 0.0
    executed = dom["exec_flops"] / sec / 1e12 if sec > 0 else 0.0
    traffic, traffic_src = profiled_traffic(wl) if tensor_kernel else (None, None)
    roofline = {"kernel": dom_name, "bound": "tensor" if tensor_kernel else "alu", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "DRAM bytes per launch", "traffic_source": traffic_src,
                "peak_source": MEASURED_BF16_SOURCE if tensor_kernel else
                "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.070 GHz",
                "algorithmic": "FP64 flops of the products the kernel computes (2 M N K each) per device time",
                "executed_tflops": executed, "executed_frac": executed / peak,
                "executed_note": "bf16 tensor flops issued: every digit pair (S(S+1)/2) over the padded tiles",
                "launches_per_step": dom["launches"], "avg_launch_ms": dom["ms"] / max(1, dom["launches"]),
                "share_of_step": sec / max(step_s, 1e-30)}
    fl = alg_flops(inst, steps)
    eff_tflops = fl["F_alg"] * value / world / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "energies/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64 (split bf16 tensor-core products)",
        "data": "synthetic (seeded: uniform orbital energies per block, symmetric Gaussian B^Q scaled by "
                "0.1 exp(-3Q/naux), random CAS CI vector with exact cumulants)",
        "config": dict(config_dict(inst, wl), precision=args.precision,
                       slices=slices if args.precision == "split" else None,
                       tuned=(not args.no_tune) and args.precision == "split"),
        "effective_tflops": eff_tflops, "flops_per_energy": fl,
        "energies": energies, "comparison": cmp, "clocks": clocks, "gpu_launches": launches,
        "roofline": roofline,
        "kernels_per_step": {k: {"launches": v["launches"], "ms": v["ms"], "flops": v["flops"],
                                 "exec_flops": v["exec_flops"]} for k, v in stats.items() if v["launches"]},
        "steps_of_energy_ms": {k: round(v["ms"], 3) for k, v in steps.items()},
        "peak_device_bytes": peak_bytes,
        "e2e": {"value": e2e_value, "unit": "energies/s", "h2d_bytes_per_step": input_bytes(inst),
                "d2h_bytes_per_step": d2h, "steps": len(e2e_ms)},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_child(wl, args.cpu_seconds)
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def scan_point_bytes(inst):
    """Device footprint of one energy of a scan point: the stored [P,P,P,H]
    class of V plus about fifteen [P,P,H,H] tensors, six spin blocks each."""
    p, h = inst["na"] + inst["nv"], inst["nc"] + inst["na"]
    return 48.0 * p ** 3 * h + 15 * 48.0 * p * p * h * h + 3e8


def scan_groups(insts, budget_bytes):
    """Indices of the points grouped into batches whose estimated footprints
    add up to at most budget_bytes (largest points first; a point larger than
    the budget gets a batch of its own)."""
    groups, cur, used = [], [], 0.0
    for k in sorted(range(len(insts)), key=lambda k: -scan_point_bytes(insts[k])):
        b = scan_point_bytes(insts[k])
        if cur and used + b > budget_bytes:
            groups.append(cur)
            cur, used = [], 0.0
        cur.append(k)
        used += b
    if cur:
        groups.append(cur)
    return groups


def run_scan(args, rank, world, local_rank):
    """The 32-point scan of uneven instances (core 4-12, CAS(4,4) or CAS(6,6),
    virtual 60-200, auxiliary 4 x virtual, virtual gap shrinking along the
    scan) through the batched call: every instance's energy captured once as
    a CUDA graph, a batch's graphs replayed at once on their own streams.
    Points are grouped into batches whose handles fit the device memory
    budget (a handle keeps its captured energy's buffers).  Ranks take
    disjoint scan points (weak scaling over points)."""
    import numpy as np
    import torch

    import paper_1701_02011_gb300 as g
    import synth
    from paper_1701_02011_gb300 import build as libbuild

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    libbuild.build()
    points = [j for j in range(32) if j % world == rank]
    insts = [synth.scan_instance(j) for j in points]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    groups = scan_groups(insts, args.scan_budget_gb * 1e9)

    def timed(prec, slices, steps):
        """Per batch: handles, one call that warms up and captures, then the
        timed replays; the batch's handles are freed before the next batch.
        A batch that runs out of device memory is halved and retried."""
        energies = [None] * len(insts)
        tot = [0.0] * steps
        launches = peak = 0
        todo = list(groups)
        done = []
        while todo:
            grp = todo.pop(0)
            devs = [{k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
                     for k, v in insts[i].items()} for i in grp]
            streams = [torch.cuda.Stream() for _ in devs]
            hs = [g.Dsrg(d, stream=st.cuda_stream, precision=prec, slices=slices,
                         tune=(not args.no_tune) and prec == g.DSRG_PREC_SPLIT) for d, st in zip(devs, streams)]
            try:
                e = g.dsrg_pt3_batch(hs)  # eager warm-up, capture, first replay
            except g.DsrgError as err:
                for h in hs:
                    h.close()
                del devs
                torch.cuda.synchronize()
                torch.cuda.empty_cache()
                if err.code != g.DSRG_ERR_OOM or len(grp) == 1:
                    raise
                todo[:0] = [grp[: len(grp) // 2], grp[len(grp) // 2:]]
                continue
            done.append(len(grp))
            for _ in range(max(args.warmup - 1, 0)):
                e = g.dsrg_pt3_batch(hs)
            for s in range(steps):
                flush.zero_()
                torch.cuda.synchronize()
                if dist:
                    dist.barrier()
                t0 = time.perf_counter()
                e = g.dsrg_pt3_batch(hs)  # host-synchronous: every energy is back on the host
                tot[s] += time.perf_counter() - t0
            for i, ei in zip(grp, e):
                energies[i] = ei
            launches += sum(g.dsrg_last_launch_count(h.h) for h in hs)
            peak = max(peak, sum(g.dsrg_peak_bytes(h.h) for h in hs))
            for h in hs:
                h.close()
            del devs
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        return energies, tot, launches, peak, done

    clocks = ClockSampler(local_rank)
    clocks.start()
    slices = args.slices or SLICES["scan32"]
    e_split, ts, launches, peak, batches = timed(g.DSRG_PREC_SPLIT, slices, args.steps)
    clk = clocks.stop()
    total_s = max_over_ranks(dist, sum(ts))
    value, tmax = aggregate([total_s], args.steps * len(points), world)
    cmp = None
    if not args.no_comparison:
        e64, ts64, _, peak64, batches64 = timed(g.DSRG_PREC_FP64, 0, 1)
        errs = {k: max(abs(a[k] - b[k]) for a, b in zip(e_split, e64)) for k in ("e2", "e3a", "e3b", "e3")}
        cmp = {"precision": "fp64", "s_per_scan": statistics.median(ts64),
               "value": len(points) / statistics.median(ts64), "max_abs_headline_minus_comparison_Eh": errs,
               "peak_bytes": peak64, "batches": batches64}
    line = {
        "metric": METRIC, "value": value, "unit": "energies/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (split bf16 tensor-core products)",
        "data": "synthetic (seeded: uniform orbital energies per block, symmetric Gaussian B^Q scaled by 0.1 exp(-3Q/naux), random CAS CI vector with exact cumulants)",
        "config": {"workload": "scan32", "instances": 32, "per_rank": len(points), "precision": "split",
                   "slices": slices, "batches": batches, "tuned": not args.no_tune,
                   "graph": "one CUDA graph per instance, a batch's graphs replayed concurrently",
                   "l2": "flushed (256 MiB write) before each timed batch"},
        "note": "a step evaluates every scan point of the rank: one batched call per memory batch, host-synchronous",
        "clocks": clk, "gpu_launches": launches * args.steps, "peak_bytes": peak, "comparison": cmp,
        "energies_e3": [e["e3"] for e in e_split],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_cholesky(args, rank, world, local_rank):
    """Pivoted incomplete Cholesky (dsrg_cholesky) of the two-electron
    supermatrix (pq|rs) = sum_Q B^Q_pq B^Q_rs of the CAS(6,6)/10 core/100
    virtual/400 aux instance (N = 116^2 = 13456 compound indices, V 1.45 GB)
    at the paper's single-point threshold 1e-6 a.u.  One step = one
    factorisation.  Roofline: HBM, algorithmic bytes per vector Q = the Q
    earlier vectors (Q N 8 B) + one row of V + the diagonal read and written
    and the vector written (4 N 8 B)."""
    import numpy as np
    import torch

    import paper_1701_02011_gb300 as g
    import synth
    from paper_1701_02011_gb300 import build as libbuild

    torch.cuda.set_device(local_rank)
    libbuild.build()
    inst = synth.config_instance("cas66_c10_v100_q400", seed=synth.config_seed("cas66_c10_v100_q400") +
                                 instance_seed_offset(rank))
    n, naux = inst["nc"] + inst["na"] + inst["nv"], inst["naux"]
    Bt = torch.from_numpy(np.ascontiguousarray(inst["B"]).reshape(naux, n * n)).cuda()
    V = (Bt.T @ Bt).contiguous()           # (pq|rs) as an N x N matrix (setup, not timed)
    del Bt
    tau, cap = 1e-6, 8 * n
    torch.cuda.synchronize()
    for _ in range(max(args.warmup, 0)):
        B, piv = g.dsrg_cholesky(V, tau, cap)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B, piv = g.dsrg_cholesky(V, tau, cap)   # host-synchronous (returns the vector count)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    nvec = len(piv)
    N = n * n
    alg_bytes = 8.0 * N * (nvec * (nvec - 1) / 2.0 + 4.0 * nvec)
    t = sum(ms) / 1000.0
    resid = float((V.diagonal() - (B * B).sum(0)).max())
    peak = _measured_hbm()
    line = {"metric": "Cholesky factorisations/s of the two-electron supermatrix (Eq. int_fact, threshold 1e-6)",
            "value": args.steps / t, "unit": "factorisations/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cholesky_cas66", "N": N, "tau": tau, "vectors": nvec,
                       "max_remaining_diagonal": resid},
            "roofline": {"bound": "hbm", "achieved": alg_bytes / (t / args.steps) / 1e9, "peak": peak[0],
                         "unit": "GB/s", "frac": alg_bytes / (t / args.steps) / 1e9 / peak[0], "traffic": None,
                         "peak_source": peak[1]},
            "clocks": clk, "gpu_launches": args.steps * (nvec + 2)}
    print(json.dumps(line), flush=True)


def run_split_gemm(args, local_rank):
    """One split-precision FP64 product C += A B (dsrg_split_gemm, the
    contraction primitive of the mixed-precision path), M = N = K = --gemm-n,
    Gaussian operands, --slices digit slices (default 8).  Packing of both
    operands included.  Roofline: the tensor pipe against the measured bf16
    peak, executed flops 2 n^3 S(S+1)/2 over the padded tiles."""
    import numpy as np
    import torch

    import paper_1701_02011_gb300 as g
    from paper_1701_02011_gb300 import build as libbuild

    torch.cuda.set_device(local_rank)
    libbuild.build()
    n, S = args.gemm_n, args.slices or 8
    rng = np.random.default_rng(0)
    A = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    B = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    for _ in range(max(args.warmup, 0)):
        g.dsrg_split_gemm(A, B, C, 1.0, S)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.dsrg_split_gemm(A, B, C, 1.0, S)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms) / 1000.0
    pad = lambda x, m: (x + m - 1) // m * m
    executed = 2.0 * pad(n, 128) * pad(n, 64) * pad(n, 16) * S * (S + 1) / 2.0
    line = {"metric": "split-precision FP64 product (M = N = K), packing included", "value": 2.0 * n ** 3 / t / 1e12,
            "unit": "TFLOP/s (FP64 products computed)", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (split bf16 tensor-core products)", "data": "synthetic (Gaussian)",
            "config": {"workload": "split_gemm", "n": n, "slices": S},
            "roofline": {"bound": "tensor", "achieved": executed / t / 1e12, "peak": MEASURED_BF16, "unit": "TFLOP/s",
                         "frac": executed / t / 1e12 / MEASURED_BF16, "traffic": None,
                         "peak_source": MEASURED_BF16_SOURCE, "algorithmic": "executed bf16 flops"},
            "gpu_launches": 3 * args.steps}
    print(json.dumps(line), flush=True)


def run_relaxed(args, rank, world, local_rank):
    """One-step relaxed DSRG-MRPT2/PT3 energies (dsrg_relaxed; Eq. E_relaxed,
    App. A) of the CAS(8,8)/30 core/300 virtual/1200 aux instance: the PT3
    energy with the all-active blocks of the summed transformed Hamiltonian,
    then the CASCI problems over its 4900 determinants (split path, 7 slices,
    tuned).  One step = one dsrg_relaxed call; the unrelaxed energy is timed
    alongside for the relaxation's cost.  Roofline: the CI matrix-vector
    product of the Lanczos iterations (HBM: the 8 ndet^2 bytes of the matrix
    and 16 ndet of the vectors per launch)."""
    import numpy as np
    import torch

    import paper_1701_02011_gb300 as g
    import synth
    from paper_1701_02011_gb300 import build as libbuild

    torch.cuda.set_device(local_rank)
    libbuild.build()
    wl = "cas88_c30_v300_q1200"
    slices = args.slices or SLICES[wl]
    inst = synth.config_instance(wl, seed=synth.config_seed(wl) + instance_seed_offset(rank))
    nel = inst["na"]
    dev = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
           for k, v in inst.items()}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    h = g.Dsrg(dev, stream=stream.cuda_stream, precision=g.DSRG_PREC_SPLIT, slices=slices, tune=not args.no_tune)
    for _ in range(max(args.warmup, 0)):
        r = h.relaxed(nel // 2, nel // 2)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = h.relaxed(nel // 2, nel // 2)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    launches = h.launches
    # the unrelaxed energy alone, and one profiled relaxed call for the matvec roofline
    with torch.cuda.stream(stream):
        flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.pt3()
    e1.record(stream)
    torch.cuda.synchronize()
    pt3_ms = e0.elapsed_time(e1)
    h.profile(True)
    h.relaxed(nel // 2, nel // 2)
    st = h.profile_stats()["k_matvec"]
    h.profile(False)
    h.close()
    t = sum(ms) / 1000.0
    peak = _measured_hbm()
    achieved = st["bytes"] / (st["ms"] / 1000.0) / 1e9 if st["ms"] > 0 else 0.0
    cmp = None
    if not args.no_comparison:
        torch.cuda.empty_cache()
        h2 = g.Dsrg(dev, stream=stream.cuda_stream)
        t0 = time.perf_counter()
        r64 = h2.relaxed(nel // 2, nel // 2)
        torch.cuda.synchronize()
        cmp = {"precision": "fp64", "seconds": time.perf_counter() - t0,
               "headline_minus_comparison_Eh": {k: r[k] - r64[k] for k in ("e2", "e3", "e_relaxed2", "e_relaxed3")}}
        h2.close()
    line = {"metric": "one-step relaxed DSRG-MRPT3 energies/s (Eq. E_relaxed)", "value": args.steps / t,
            "unit": "energies/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (split bf16 tensor-core products, FP64 CI)", "data": "synthetic",
            "config": {"workload": "relaxed_cas88_c30_v300_q1200", "slices": slices, "ndet": r["ndet"],
                       "l2_flush": "256 MiB write before each step"},
            "energies": {k: r[k] for k in ("e2", "e3", "e_relaxed2", "e_relaxed3", "residual2", "residual3",
                                           "steps2", "steps3")},
            "unrelaxed_ms": pt3_ms, "relaxation_ms": 1000.0 * t / args.steps - pt3_ms,
            "comparison": cmp,
            "roofline": {"bound": "hbm", "kernel": "k_matvec", "achieved": achieved, "peak": peak[0], "unit": "GB/s",
                         "frac": achieved / peak[0], "traffic": None, "peak_source": peak[1],
                         "launches": st["launches"], "ms": st["ms"]},
            "clocks": clk, "gpu_launches": launches * args.steps}
    print(json.dumps(line), flush=True)


def run_dyall(args, rank, world, local_rank):
    """First-order aavv amplitudes with Dyall's H(0) at s -> infinity
    (dsrg_dyall_aavv; App. B, Eq. t2_aavv) on the CAS(8,8)/30 core/300
    virtual/1200 aux instance: 360000 virtual spin-orbital pairs x 256 active
    pairs, split path (7 slices).  One step = one call (iterate to 1e-10 of
    max |V|, or until the residual diverges on small shifted denominators,
    the intruders of App. B: the synthetic virtual band starts below the top
    of the active one); the rate is Jacobi iterations per second and the
    result reports convergence and the denominator statistics.
    Roofline: the element-wise Jacobi update (HBM: V, the product and the
    amplitudes read, the amplitudes written, 32 B per element per
    iteration) and the coupling product on the tensor cores."""
    import numpy as np
    import torch

    import paper_1701_02011_gb300 as g
    import synth
    from paper_1701_02011_gb300 import build as libbuild

    torch.cuda.set_device(local_rank)
    libbuild.build()
    wl = "cas88_c30_v300_q1200"
    slices = args.slices or SLICES[wl]
    inst = synth.config_instance(wl, seed=synth.config_seed(wl) + instance_seed_offset(rank))
    dev = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
           for k, v in inst.items()}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    h = g.Dsrg(dev, stream=stream.cuda_stream, precision=g.DSRG_PREC_SPLIT, slices=slices, tune=not args.no_tune)
    for _ in range(max(args.warmup, 0)):
        r = h.dyall_aavv(1e-10, 300)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = h.dyall_aavv(1e-10, 300)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    launches = h.launches
    h.profile(True)
    h.dyall_aavv(1e-10, 300)
    st = h.profile_stats()
    h.profile(False)
    h.close()
    t = sum(ms) / 1000.0
    peak = _measured_hbm()
    upd, mma = st["k_amp"], st["k_ozaki_mma"]
    upd_gbs = upd["bytes"] / (upd["ms"] / 1000.0) / 1e9 if upd["ms"] > 0 else 0.0
    mma_tf = mma["exec_flops"] / (mma["ms"] / 1000.0) / 1e12 if mma["ms"] > 0 else 0.0
    hbm_dominant = upd["ms"] >= mma["ms"]
    roof = ({"bound": "hbm", "kernel": "k_dy_update", "achieved": upd_gbs, "peak": peak[0], "unit": "GB/s",
             "frac": upd_gbs / peak[0], "traffic": None, "peak_source": peak[1]} if hbm_dominant else
            {"bound": "tensor", "kernel": "k_ozaki_mma", "achieved": mma_tf, "peak": MEASURED_BF16,
             "unit": "TFLOP/s", "frac": mma_tf / MEASURED_BF16, "traffic": None, "peak_source": MEASURED_BF16_SOURCE,
             "algorithmic": "executed bf16 flops"})
    roof["kernel_ms"] = {"k_dy_update": upd["ms"], "k_ozaki_mma": mma["ms"], "k_ozaki_pack": st["k_ozaki_pack"]["ms"]}
    iters = r["iterations"] * args.steps
    line = {"metric": "Dyall-H(0) aavv Jacobi iterations/s (Eq. t2_aavv, s -> infinity)", "value": iters / t,
            "unit": "iterations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (split bf16 tensor-core products)", "data": "synthetic",
            "config": {"workload": "dyall_cas88_c30_v300_q1200", "slices": slices, "tol": 1e-10,
                       "unknowns": 4 * inst["nv"] ** 2 * 4 * inst["na"] ** 2,
                       "l2_flush": "256 MiB write before each step"},
            "result": r, "roofline": roof, "clocks": clk, "gpu_launches": launches * args.steps}
    print(json.dumps(line), flush=True)


def _measured_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "of measured"
    return 6800.0, "of fallback"


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="oracle rows timed for the cpu_baseline (at least one row)")
    ap.add_argument("--ref-rows", type=int, default=1, help="oracle ladder rows per step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=("split", "fp64"), default="split",
                    help="headline path; the other is timed on one energy alongside for comparison")
    ap.add_argument("--slices", type=int, default=0, help="digit slices of the split path (0: per workload)")
    ap.add_argument("--e2e-steps", type=int, default=2, help="end-to-end energies timed (at most --steps)")
    ap.add_argument("--no-comparison", action="store_true",
                    help="skip timing the other precision (quick runs, profiler launch lists)")
    ap.add_argument("--no-tune", action="store_true",
                    help="fixed tile/split rules for the split products (default: tuned in the first warm-up)")
    ap.add_argument("--workload", choices=("cas88_c30_v300_q1200", "cas66_c10_v100_q400", "cas44_c40_v500_q1800",
                                           "scan32", "cas1616_c10_v100_q400", "cholesky_cas66", "split_gemm",
                                           "relaxed_cas88_c30_v300_q1200", "dyall_cas88_c30_v300_q1200"),
                    default=WORKLOAD,
                    help="CAS(8,8)/30 core/300 virtual (default), CAS(6,6)/10 core/100 virtual, "
                         "CAS(4,4)/40 core/500 virtual, the batched 32-point scan, a synthetic 16-orbital active "
                         "space (10 core, 100 virtual), the Cholesky factorisation of the CAS(6,6)-size "
                         "two-electron supermatrix, one split-precision product (--gemm-n), or the one-step "
                         "relaxed energies of the CAS(8,8) instance, or its Dyall-H(0) aavv amplitudes")
    ap.add_argument("--gemm-n", type=int, default=4096, help="split_gemm: M = N = K")
    ap.add_argument("--scan-budget-gb", type=float, default=250.0,
                    help="device memory per scan batch (handles keep their captured buffers)")
    args = ap.parse_args(argv)
    rank, world, local_rank = rank_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "scan32":
        run_scan(args, rank, world, local_rank)
    elif args.workload == "cholesky_cas66":
        run_cholesky(args, rank, world, local_rank)
    elif args.workload == "split_gemm":
        run_split_gemm(args, local_rank)
    elif args.workload == "relaxed_cas88_c30_v300_q1200":
        run_relaxed(args, rank, world, local_rank)
    elif args.workload == "dyall_cas88_c30_v300_q1200":
        run_dyall(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
