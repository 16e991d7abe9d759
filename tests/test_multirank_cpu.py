"""The multi-process path of bench.py on CPU: two gloo ranks, as torchrun
would launch them.  The data path has no collective (each rank advances its
own seeded copy of the workload); the only exchange is the max over ranks of
the timed seconds, and the reported value is the whole job's throughput."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    t = bench.max_over_ranks(1.0 + rank, dist)       # rank 1 is the slower one
    dist.barrier()
    out[rank] = (r, w, local, t)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == (0, 2, 0, 2.0)
    assert res[1] == (1, 2, 1, 2.0)


def test_weak_scaling_value_counts_every_rank():
    import bench
    one = bench.node_updates_per_s(16384, 20, 1, 9, 0.5)
    two = bench.node_updates_per_s(16384, 20, 2, 9, 0.5)
    assert one == 16384 * 20 * 11 / 0.5
    assert two == 2 * one


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    # a rank other than 0 returns at once, before reading its arguments or
    # touching the oracle
    assert bench.run_reference(None, 1) is None
    assert capsys.readouterr().out == ""


def test_step_counters_cover_the_default_bench_modes():
    """The default bench workload's headline mode and its float-float
    variant have a line in profiles/step_counters.txt (the ALU roof's
    executed FLOP and the measured DRAM traffic)."""
    import bench
    for mode in ("fp64", "fp32"):
        c = bench.step_counters("tube", mode)
        assert c is not None, mode
        key = "fp64_flop" if mode == "fp64" else "fp32_flop"
        assert c[key] > 1000 and c["dram_bytes"] > 0
