"""The multi-GPU form is replicas only (one instance per rank, no collective on the data path):
the bench's rank-to-instance mapping and its max-over-ranks timing, run as two gloo ranks on CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2206_11009_gb300 import synth
    seed = bench.rank_instance_seed(rank)
    inst = synth.image_pair(8, seed)
    t = bench.max_over_ranks(1.0 + rank, world)
    bench.barrier(world)
    out.put((rank, seed, float(inst.a.sum()), t))
    dist.destroy_process_group()


def test_two_ranks_distinct_instances_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, t0), (r1, s1, m1, t1) = res
    assert (r0, r1) == (0, 1) and s0 != s1          # each rank its own instance
    assert abs(m0 - 1.0) < 1e-12 and abs(m1 - 1.0) < 1e-12
    assert t0 == t1 == 2.0                         # both report the slowest rank's time
