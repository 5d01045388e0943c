"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

The path shards by shots: every rank inverts its own shot of the same sizes
(seed = rank) with no data-path collective; the ranks meet only for the
timing (a barrier and the maximum over ranks), and the job's value is all
ranks' cells over the slowest rank's time.  The reference arm runs on rank 0
only; other ranks return without work.
"""
import io
import os
import socket
import contextlib

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        w = bench.rank_workload("c1", rank)
        shape = torch.tensor([w.nr, w.nz, w.nt, len(w.shots)], dtype=torch.int64)
        shapes = [torch.zeros_like(shape) for _ in range(world)]
        dist.all_gather(shapes, shape)
        vsum = torch.tensor([float(w.vp.astype("float64").sum())], dtype=torch.float64)
        vsums = [torch.zeros_like(vsum) for _ in range(world)]
        dist.all_gather(vsums, vsum)
        ms = bench.max_over_ranks(10.0 + 2.5 * rank, world)
        rate = bench.job_rate(3.0e9, world, ms)
        printed = ""
        if rank > 0:
            # the reference arm does no work off rank 0
            args = bench.parse_args(["--impl", "reference", "--gpus", str(world)])
            buf = io.StringIO()
            with contextlib.redirect_stdout(buf):
                bench.run_reference(args, w)
            printed = buf.getvalue()
        dist.barrier()
        q.put((rank, [s.tolist() for s in shapes], [float(v) for v in vsums], ms, rate, printed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            rank, shapes, vsums, ms, rate, printed = q.get(timeout=240)
            out[rank] = (shapes, vsums, ms, rate, printed)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    for rank in (0, 1):
        shapes, vsums, ms, rate, printed = out[rank]
        assert shapes[0] == shapes[1]            # same sizes on every rank
        assert vsums[0] != vsums[1]              # independent models (seed = rank)
        assert ms == 12.5                        # the slowest rank's time
        assert rate == pytest.approx(2 * 3.0e9 / 12.5e-3 / 1e9)
    assert out[1][4] == ""
