#!/usr/bin/env python
"""DSRG-MRPT3 energy throughput on GB300.

One step = one full unrelaxed DSRG-MRPT3 energy (first-order amplitudes,
E(2), the second-order transformed Hamiltonian with the density-fitted
particle-particle ladder, second-order amplitudes, E(3)) of the synthetic
workload below, through the library's C interface.

Workload (default): 10 core, CAS(6,6) reference (400 Ms=0 determinants,
seeded random CI vector with exact gamma1 / lambda2 / lambda3), 100 virtual,
400 auxiliary functions, s = 0.5 Eh^-2; orbital energies and B^Q_pq drawn as
described in the design doc.  Inputs are smaller than L2, so L2 is flushed
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


def config_dict(inst, precision):
    return {"workload": WORKLOAD, "nc": inst["nc"], "na": inst["na"], "nv": inst["nv"], "naux": inst["naux"],
            "s": inst["s"], "precision": precision, "l2": "flushed (256 MiB write) before each timed step",
            "reference": "CAS(6,6) Ms=0, 400 determinants"}


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
    inst = synth.config_instance(WORKLOAD, seed=synth.CONFIGS[WORKLOAD]["seed"] + instance_seed_offset(rank))
    stream = torch.cuda.Stream()
    dev = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
           for k, v in inst.items()}
    torch.cuda.synchronize()
    h = g.Dsrg(dev, stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    energies = None
    for _ in range(max(args.warmup, 0)):
        energies = h.pt3()
    # ---- timed region: inputs resident on the device
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank)
    clk.start()
    h.profile(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            starts[k].record(stream)
        energies = h.pt3()
        launches += h.launches
        with torch.cuda.stream(stream):
            ends[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    stats = h.profile_stats()
    h.profile(False)
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = sum(ms) / 1000.0
    if dist:
        t = torch.tensor([total_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value, tmax = aggregate([total_s], args.steps, world)
    ms_per_step = 1000.0 * tmax / args.steps
    # ---- end to end: host buffers (pinned), copies inside the timed region
    host = {}
    for k, v in inst.items():
        if isinstance(v, np.ndarray):
            t = torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
            host[k] = t.numpy()
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
        e = h.pt3()
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
        d2h = g.dsrg_last_d2h_bytes(h.h) + 32
    e2e_value = world * 1000.0 / statistics.median(e2e_ms)
    # ---- roofline of the dominant kernel
    dom = max(stats.items(), key=lambda kv: kv[1]["ms"])
    fp64_peak = FP64_ALU_PEAK_TFLOPS
    peak_src = "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.070 GHz"
    af = alg_flops(inst)
    name, st = dom
    if name == "k_gemm<1>":
        alg = af["build"] * args.steps
        alg_note = "Q p^2 (p^2+1) per energy ((pr|qs) build, pair-swap symmetry)"
    elif name == "k_gemm<2>":
        alg = af["ladder"] * args.steps
        alg_note = "h (h+1) p^4 per energy (ladder, i <= j)"
    else:
        alg = st["flops"]
        alg_note = "2 M N K summed over the kernel's contractions"
    achieved = alg / (st["ms"] / 1000.0) / 1e12 if st["ms"] > 0 else 0.0
    roofline = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": None, "peak_source": peak_src,
                "algorithmic": alg_note, "launches_per_step": st["launches"] / args.steps,
                "avg_launch_ms": st["ms"] / max(1, st["launches"]),
                "share_of_step": (st["ms"] / 1000.0) / max(total_s, 1e-30)}
    eff_tflops = (af["ladder"] + af["build"]) * value / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "energies/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded; see DESIGN.md)",
        "config": config_dict(inst, "fp64"),
        "effective_tflops_ladder_build": eff_tflops,
        "energies": energies,
        "clocks": clocks,
        "gpu_launches": launches,
        "roofline": roofline,
        "kernels": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in stats.items()},
        "e2e": {"value": e2e_value, "unit": "energies/s", "h2d_bytes_per_step": input_bytes(inst),
                "d2h_bytes_per_step": d2h},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, t, text = oracle_sample_rate(inst, args.cpu_reps)
        line["cpu_baseline"] = {"value": cb, "unit": "energies/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": text}
    elif rank == 0:
        line["cpu_baseline"] = None
    h.close()
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
    args = ap.parse_args(argv)
    rank, world, local_rank = rank_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
