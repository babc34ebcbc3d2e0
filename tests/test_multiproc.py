"""The multi-GPU host logic of bench.py on CPU: two gloo ranks (no GPU).

The binaries are independent, so ranks never exchange data: each rank gets its
own seeded ensemble, and only the timing is reduced (max over ranks) to form the
whole-job rate.  Here each rank integrates a small shard with the CPU oracle in
place of the GPU work.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import time

    import torch
    import torch.distributed as dist

    import bench
    import oracle
    import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    seed = bench.rank_seed(r)
    ens = workloads.config("C1", n=64, seed=seed)
    t0 = time.perf_counter()
    out = oracle.integrate(ens, threads=1)
    ms = (time.perf_counter() - t0) * 1e3 + (50.0 if r == 1 else 0.0)
    mx = bench.reduce_max(ms, dist, torch.device("cpu"))
    seeds = [None] * w
    dist.all_gather_object(seeds, seed)
    q.put((r, w, lr, seed, float(out["t"].sum()), ms, mx, seeds, bench.aggregate_rate(w, 64, 1, mx)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_exchange():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, t0, ms0, mx0, seeds0, rate0), (r1, w1, l1, s1, t1, ms1, mx1, seeds1, rate1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert s0 != s1 and seeds0 == seeds1 == [s0, s1]       # distinct shards, agreed by both ranks
    assert t0 != t1                                        # different binaries integrated
    assert mx0 == mx1 == pytest.approx(max(ms0, ms1))      # timing: max over ranks
    assert rate0 == rate1 == pytest.approx(2 * 64 / (mx0 * 1e-3))


# ---------------------------------------------------------------------------
# Failure detection on the host.  The ranks share nothing but the timing
# reduction and the barriers, so a failed rank must surface on the others as an
# error from their next collective (or from the rendezvous), not as a wait without
# end.  The failures are made on the host: a rank that raises, one that never
# joins, one that leaves between steps.

def _fail_worker(rank, world, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import time

    import torch

    import bench
    t0 = time.perf_counter()
    try:
        if mode == "never_joins" and rank == 1:
            q.put((rank, "absent", 0.0))
            return
        tdist = bench.init_dist("gloo", timeout_s=4.0)
        if mode == "raises" and rank == 1:
            raise RuntimeError("injected failure before the timing reduction")
        if mode == "leaves" and rank == 1:
            bench.reduce_max(1.0, tdist, torch.device("cpu"))   # step 1 completes on both ranks
            q.put((rank, "left", time.perf_counter() - t0))
            q.close()
            q.join_thread()                                     # flush the report before leaving
            os._exit(0)                                         # leaves between steps, no teardown
        bench.reduce_max(1.0, tdist, torch.device("cpu"))
        if mode == "leaves":
            time.sleep(0.5)
            tdist.barrier()                                     # step 2: the peer is gone
        q.put((rank, "ok", time.perf_counter() - t0))
        tdist.destroy_process_group()
    except RuntimeError as e:       # torch.distributed errors derive from RuntimeError
        q.put((rank, "error:" + type(e).__name__, time.perf_counter() - t0))


def _run_failure_case(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_fail_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, what, dt = q.get(timeout=120)
        res[r] = (what, dt)
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():            # only the process this test started
            p.kill()
            p.join()
    return res


@pytest.mark.parametrize("mode,peer", [("raises", "error:RuntimeError"), ("never_joins", "absent"),
                                       ("leaves", "left")])
def test_failed_rank_surfaces_as_an_error_on_the_other(mode, peer):
    res = _run_failure_case(mode)
    what0, dt0 = res[0]
    assert what0.startswith("error:"), res       # rank 0 learns of the failure ...
    assert dt0 < 60.0, res                       # ... within the bounded timeout, not never
    assert res[1][0] == peer, res
