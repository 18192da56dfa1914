"""The benchmark's multi-rank host logic on CPU: two gloo ranks.

bench.py under torchrun runs one replica per GPU; its timing is the maximum
over ranks and its throughput the sum of all ranks' pairs over that time.
Here two CPU processes join a gloo group through the same set-up code and
check the reductions, the barrier, and that only rank 0 runs the reference
arm (the other ranks return at once).
"""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    w, r, _ = bench.dist_setup(None)
    try:
        bench.barrier(w)
        mx = bench.max_over_ranks(float(r + 1), w)
        sm = bench.sum_over_ranks(float(10 * (r + 1)), w)
        ref = bench.run_reference(None, w, r) if r != 0 else "skipped"
        bench.barrier(w)
        q.put((r, w, dist.get_backend(), mx, sm, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, backend, mx, sm, ref in out:
        assert w == 2 and backend == "gloo"
        assert mx == 2.0 and sm == 30.0
    assert out[1][5] is None            # rank 1 does no reference work
