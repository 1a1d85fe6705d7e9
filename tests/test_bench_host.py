"""Host logic of the multi-GPU bench (one instance per rank, weak scaling):
two gloo ranks on the CPU run the same reduction the GPU ranks run over NCCL."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.rank_env()
    seconds = 1.0 + 0.5 * r  # rank 1 is the slow one
    t = bench.max_over_ranks(dist, seconds, device="cpu")
    value, tmax = bench.aggregate([t], 5, w)
    inst = synth.config_instance("cas44_c2_v12_q60",
                                 seed=synth.CONFIGS["cas44_c2_v12_q60"]["seed"] + bench.instance_seed_offset(r))
    out[r] = (r, w, lr, t, value, tmax, float(np.asarray(inst["B"]).sum()))
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = [out[r] for r in range(world)]
    for r, (rr, w, lr, t, value, tmax, bsum) in enumerate(res):
        assert (rr, w, lr) == (r, world, r)
        assert t == pytest.approx(1.5)  # max over ranks, seen by every rank
        assert tmax == pytest.approx(1.5)
        assert value == pytest.approx(world * 5 / 1.5)  # all ranks' energies / slowest time
    # every rank evaluates its own instance of the same sizes
    assert res[0][6] != res[1][6]


def test_aggregate_single_rank():
    v, t = bench.aggregate([2.0], 4, 1)
    assert (v, t) == (2.0, 2.0)
    assert bench.instance_seed_offset(0) == 0 and bench.instance_seed_offset(3) == 3000


def test_scan_groups_cover_every_point_within_budget():
    insts = [synth.scan_sizes(j) for j in range(32)]
    sizes = [bench.scan_point_bytes(i) for i in insts]
    for budget in (3e11, 1.2e11, 4e10, 1.0):
        groups = bench.scan_groups(insts, budget)
        flat = sorted(k for g in groups for k in g)
        assert flat == list(range(32))  # every point exactly once
        for g in groups:
            assert len(g) == 1 or sum(sizes[k] for k in g) <= budget
    assert len(bench.scan_groups(insts, 3e11)) == 1
    assert all(len(g) == 1 for g in bench.scan_groups(insts, 1.0))


def test_profiled_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu summary only while the
    split kernel's source is the one the counters were taken on."""
    import shutil
    wl = "cas88_c30_v300_q1200"
    traffic, src = bench.profiled_traffic(wl)
    assert traffic is not None and traffic > 0, src
    assert src == f"profiles/k_ozaki_mma_{wl}.md"
    # a copy of the tree whose kernel source differs by one byte
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_1701_02011_gb300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", f"k_ozaki_mma_{wl}.md"), tmp_path / "profiles")
    kernel = open(os.path.join(bench.ROOT, "paper_1701_02011_gb300", "csrc", "ozaki.cu"), "rb").read()
    (csrc / "ozaki.cu").write_bytes(kernel)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic(wl)[0] == traffic
    (csrc / "ozaki.cu").write_bytes(kernel + b"\n")
    t2, why = bench.profiled_traffic(wl)
    assert t2 is None and "predates" in why
    assert bench.profiled_traffic("no_such_workload") == (None, None)
