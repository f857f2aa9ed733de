"""Multi-rank host logic of bench.py (one replica per rank, max-over-ranks timing),
exercised with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.allreduce_max(1.0 + rank)           # rank r measured 1 + r seconds
        out[rank] = (t, bench.aggregate_mlups(1_000_000, 10, world, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_work():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == (2.0, pytest.approx(2 * 1_000_000 * 10 / 2.0 / 1e6))


def test_single_process_is_its_own_max():
    import bench
    assert bench.allreduce_max(3.5) == 3.5
    assert bench.aggregate_mlups(100, 10, 1, 0.5) == pytest.approx(100 * 10 / 0.5 / 1e6)


def test_reference_arm_times_oracle_steps_within_budget():
    """The reference arm (the oracle on the host cores) sizes its slab so that the run
    fits the time budget and reports the keys the bench line carries."""
    import time

    import bench
    t0 = time.perf_counter()
    cpu = bench.reference_steps(2, 1, budget_s=2.0)
    # the stepped part (1 warm-up + 2 timed oracle steps) keeps to the budget (the slab is
    # at least one plane thick); the synthetic input field itself takes longer to make
    assert 3 * cpu["ms_per_step"] / 1e3 < 4 * 2.0
    assert time.perf_counter() - t0 < 300.0
    for key in ("value", "unit", "cores", "kind", "sample", "ms_per_step"):
        assert key in cpu
    assert cpu["kind"] == "oracle" and cpu["unit"] == "MLUPS" and cpu["value"] > 0 and cpu["cores"] >= 1
