#!/usr/bin/env python
"""DSRG-MRPT3 energy throughput on GB300.

One step = one full unrelaxed DSRG-MRPT3 energy (first-order amplitudes,
E(2), the second-order transformed Hamiltonian with the density-fitted
particle-particle ladder, second-order amplitudes, E(3)) of the synthetic
workload below, through the library's C interface.

Workload (default): 10 core, CAS(6,6) reference (400 Ms=0 determinants,
seeded random CI vector with exact gamma1 / lambda2 / lambda3), 100 virtual,
400 auxiliary functions, s = 0.5 Eh^-2; orbital energies and B^Q_pq drawn as
drawn from the seeded generator in synth/.  Inputs are smaller than L2, so L2 is flushed
(a 256 MiB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
WORKLOAD = "cas66_c10_v100_q400"
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

def profiled_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu launch list of
    the split path on `workload` (profiles/launches_split_<workload>.md: one
    energy, dram__bytes_read.sum + dram__bytes_write.sum), or None."""
    path = os.path.join(ROOT, "profiles", f"launches_split_{workload}.md")
    if not os.path.exists(path):
        return None, None
    prefix = {"k_ozaki_mma": ("k_ozaki_mma<",), "k_gemm<0>": ("k_gemm_flat<", "k_gemm<64, 64, 0>")}.get(kernel)
    if not prefix:
        return None, None
    launches = gb = 0.0
    for line in open(path):
        cells = [c.strip().strip("`") for c in line.strip().strip("|").split("|")]
        if len(cells) >= 5 and cells[0].startswith(prefix):
            try:
                launches += float(cells[1])
                gb += float(cells[4])
            except ValueError:
                pass
    if not launches:
        return None, None
    return gb * 1e9 / launches, (f"profiles/launches_split_{workload}.md (per-launch mean over one energy of the "
                                 "--no-tune run: under ncu's serialised launches the tuner's timings are skewed)")

SAMPLE_WORKLOAD = "cas44_c2_v12_q60"


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

def _nso(inst):
    return 2 * (inst["nc"] + inst["na"] + inst["nv"])


def oracle_sample_rate(target_inst, reps: int):
    """Time the oracle as it stands on the small CAS(4,4) instance and scale
    by its dense O(n_so^6) cost to the target size.  Returns
    (energies_per_s at target size, seconds per sample, sample text)."""
    import synth
    from oracle import dsrg as odsrg
    inst = synth.config_instance(SAMPLE_WORKLOAD)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        odsrg.dsrg_pt3(inst)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    scale = (_nso(target_inst) / _nso(inst)) ** 6
    text = (f"full PT3 oracle evaluation of the CAS(4,4), 2 core, 12 virtual, 60 aux instance "
            f"({_nso(inst)} spin orbitals), median of {reps}, scaled by the oracle's dense O(n_so^6) "
            f"cost to {_nso(target_inst)} spin orbitals (x{scale:.3g})")
    return 1.0 / (t * scale), t, text


# ----------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return
    import synth
    target = synth.config_instance(WORKLOAD)
    for _ in range(args.warmup):
        oracle_sample_rate(target, 1)
    rates, secs = [], []
    text = ""
    for _ in range(args.steps):
        r, t, text = oracle_sample_rate(target, 1)
        rates.append(r)
        secs.append(t)
    value = statistics.median(rates)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "energies/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(target, "fp64 CPU oracle"),
        "cpu_baseline": {"value": value, "unit": "energies/s", "cores": cores, "kind": "oracle",
                         "sample": text},
        "e2e": {"value": value, "unit": "energies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(inst, precision, workload=WORKLOAD):
    na = inst["na"]
    from math import comb
    dets = comb(na, na // 2) ** 2
    return {"workload": workload, "nc": inst["nc"], "na": na, "nv": inst["nv"], "naux": inst["naux"],
            "s": inst["s"], "precision": precision, "l2": "flushed (256 MiB write) before each timed step",
            "reference": f"CAS({na},{na}) Ms=0, {dets} determinants"}


def input_bytes(inst):
    import numpy as np
    tot = 0
    for k in ("eps", "B", "g1a", "g1b", "l2aa", "l2ab", "l2bb", "l3aaa", "l3aab", "l3abb", "l3bbb"):
        tot += np.asarray(inst[k]).nbytes
    return tot


def alg_flops(inst):
    """Algorithmic flop counts of the dense contractions of one PT3 energy.

    ladder over particle pairs i <= j: h(h+1) p^4; (pr|qs) build with the
    pair-swap symmetry: Q p^2 (p^2 + 1); p = active + virtual, h = core + active.
    """
    h = inst["nc"] + inst["na"]
    p = inst["na"] + inst["nv"]
    Q = inst["naux"]
    return {"ladder": h * (h + 1) * p ** 4, "build": Q * p * p * (p * p + 1)}


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
    # one profiled energy: per-kernel device time, launches and flops of a step
    stats = {}
    if profile:
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        h.profile(True)
        h.pt3()
        torch.cuda.synchronize()
        stats = h.profile_stats()
        h.profile(False)
    return h, ms, energies, stats, launches, clk


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
    inst = synth.config_instance(wl, seed=synth.CONFIGS[wl]["seed"] + instance_seed_offset(rank))
    stream = torch.cuda.Stream()
    dev = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
           for k, v in inst.items()}
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    other = "fp64" if args.precision == "split" else "split"
    # comparison path first (untimed for the headline), then the headline path
    ms2 = e_other = None
    if not args.no_comparison:
        # context and accuracy reference only: one warm-up, one timed energy
        h2, ms2, e_other, stats2, _, _ = _time_path(g, torch, dev, stream, flush, 1, 1, other, args.slices,
                                                    tune=not args.no_tune, profile=False)
        h2.close()
    if dist:
        dist.barrier()
    h, ms, energies, stats, launches, clocks = _time_path(g, torch, dev, stream, flush, args.steps, args.warmup,
                                                          args.precision, args.slices, ClockSampler(local_rank),
                                                          tune=not args.no_tune)
    if dist:
        dist.barrier()
    total_s = max_over_ranks(dist, sum(ms) / 1000.0)
    value, tmax = aggregate([total_s], args.steps, world)
    ms_per_step = 1000.0 * tmax / args.steps
    # ---- end to end: host buffers (pinned), copies inside the timed region
    host = {}
    for k, v in inst.items():
        if isinstance(v, np.ndarray):
            host[k] = torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()
        else:
            host[k] = v
    e2e_ms = []
    d2h = 0
    for k in range(max(1, min(args.steps, 5))):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.load(host)
        h.pt3()
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
        d2h = g.dsrg_last_d2h_bytes(h.h) + 32
    e2e_value = world * 1000.0 / statistics.median(e2e_ms)
    h.close()
    # ---- roofline of the dominant kernel (by device time in the profiled energy)
    dom_name, dom = max(stats.items(), key=lambda kv: kv[1]["ms"])
    af = alg_flops(inst)
    step_s = total_s / args.steps
    if dom_name == "k_gemm<1>":
        alg, note = af["build"], "Q p^2 (p^2+1) per energy ((pr|qs) build, pair-swap symmetry)"
    elif dom_name == "k_gemm<2>":
        alg, note = af["ladder"], "h (h+1) p^4 per energy (ladder, i <= j)"
    elif dom_name == "k_ozaki_mma":
        alg, note = dom["flops"], "executed bf16 flops: 2 x 128-row x tile-width x 64-k tiles x S(S+1)/2 digit pairs"
    else:
        alg, note = dom["flops"], "2 M N K summed over the kernel's contractions"
    tensor_kernel = dom_name == "k_ozaki_mma"
    peak = MEASURED_BF16 if tensor_kernel else FP64_ALU_PEAK_TFLOPS
    achieved = alg / (dom["ms"] / 1000.0) / 1e12 if dom["ms"] > 0 else 0.0
    traffic, traffic_src = profiled_traffic(dom_name, wl) if args.precision == "split" else (None, None)
    roofline = {"kernel": dom_name, "bound": "tensor" if tensor_kernel else "alu", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch", "traffic_source": traffic_src,
                "peak_source": MEASURED_BF16_SOURCE if tensor_kernel else
                "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.070 GHz",
                "algorithmic": note, "launches_per_step": dom["launches"],
                "avg_launch_ms": dom["ms"] / max(1, dom["launches"]),
                "share_of_step": (dom["ms"] / 1000.0) / max(step_s, 1e-30)}
    tensor = stats.get("k_ozaki_mma", {"launches": 0, "ms": 0.0, "flops": 0.0})
    roof_tensor = None
    if tensor["launches"] and dom_name != "k_ozaki_mma":
        executed = tensor["flops"] / (tensor["ms"] / 1000.0) / 1e12
        roof_tensor = {"kernel": "k_ozaki_mma", "bound": "tensor", "achieved": executed, "peak": MEASURED_BF16,
                       "unit": "TFLOP/s", "frac": executed / MEASURED_BF16,
                       "note": "executed bf16 flops (digit-slice pairs and tile padding included) per device time",
                       "launches_per_step": tensor["launches"],
                       "share_of_step": (tensor["ms"] / 1000.0) / max(step_s, 1e-30)}
    fp64k = stats.get("k_gemm<0>", {"launches": 0, "ms": 0.0, "flops": 0.0})
    roof_fp64 = None
    if fp64k["launches"] and dom_name != "k_gemm<0>":
        a64 = fp64k["flops"] / (fp64k["ms"] / 1000.0) / 1e12
        roof_fp64 = {"kernel": "k_gemm<0>", "bound": "alu", "achieved": a64, "peak": FP64_ALU_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": a64 / FP64_ALU_PEAK_TFLOPS,
                     "note": "2 M N K of the FP64 contractions per device time",
                     "launches_per_step": fp64k["launches"],
                     "share_of_step": (fp64k["ms"] / 1000.0) / max(step_s, 1e-30)}
    eff_tflops = (af["ladder"] + af["build"]) * value / 1e12
    err = {k: energies[k] - e_other[k] for k in ("e2", "e3a", "e3b", "e3")} if e_other else None
    line = {
        "metric": METRIC, "value": value, "unit": "energies/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64 (split bf16 tensor-core products)",
        "data": "synthetic (seeded: uniform orbital energies per block, symmetric Gaussian B^Q scaled by 0.1 exp(-3Q/naux), random CAS CI vector with exact cumulants)",
        "config": dict(config_dict(inst, args.precision, wl), slices=args.slices if args.precision == "split" else None,
                       tuned=(not args.no_tune) and args.precision == "split"),
        "effective_tflops_ladder_build": eff_tflops,
        "energies": energies,
        "comparison": None if ms2 is None else
        {"precision": other, "ms_per_step": statistics.median(ms2), "value": 1000.0 / statistics.median(ms2),
         "energies": e_other, "headline_minus_comparison_Eh": err},
        "clocks": clocks,
        "gpu_launches": launches,
        "roofline": roofline,
        "roofline_tensor": roof_tensor,
        "roofline_fp64": roof_fp64,
        "kernels_per_step": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in stats.items() if v["launches"]},
        "e2e": {"value": e2e_value, "unit": "energies/s", "h2d_bytes_per_step": input_bytes(inst),
                "d2h_bytes_per_step": d2h},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, t, text = oracle_sample_rate(inst, args.cpu_reps)
        line["cpu_baseline"] = {"value": cb, "unit": "energies/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": text}
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
    e_split, ts, launches, peak, batches = timed(g.DSRG_PREC_SPLIT, args.slices, args.steps)
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
                   "slices": args.slices, "batches": batches, "tuned": not args.no_tune,
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


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-reps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=("split", "fp64"), default="split",
                    help="headline path; the other is timed alongside for comparison")
    ap.add_argument("--slices", type=int, default=6)
    ap.add_argument("--no-comparison", action="store_true",
                    help="skip timing the other precision (quick runs, profiler launch lists)")
    ap.add_argument("--no-tune", action="store_true",
                    help="fixed tile/split rules for the split products (default: tuned in the first warm-up)")
    ap.add_argument("--workload", choices=("cas66_c10_v100_q400", "cas88_c30_v300_q1200", "cas44_c40_v500_q1800",
                                           "scan32"),
                    default=WORKLOAD,
                    help="the CAS(6,6) instance (default), the CAS(8,8)/300-virtual or CAS(4,4)/500-virtual "
                         "instances (use --slices 8), or the batched 32-point scan")
    ap.add_argument("--scan-budget-gb", type=float, default=250.0,
                    help="device memory per scan batch (handles keep their captured buffers)")
    args = ap.parse_args(argv)
    rank, world, local_rank = rank_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "scan32":
        run_scan(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
