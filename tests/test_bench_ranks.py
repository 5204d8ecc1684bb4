"""The replica (weak-scaling) aggregation of bench.py across ranks, on CPU with
gloo and world size 2: every rank reports the units of all ranks over the
slowest rank's time."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [0.5, 2.0][rank]            # rank 1 is the slow one
        rate, worst = bench.job_rate(local, 1000, world, "cpu", dist)
        out[rank] = (rate, worst)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_rate_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (1000 * 2 / 2.0, 2.0)


def test_job_rate_single_rank():
    import bench
    assert bench.job_rate(0.25, 100, 1) == (400.0, 0.25)


def test_step_byte_model():
    """The whole-step byte model: 15 B per particle (8-bit velocities) + 40 B per
    cell of 64 tiles of 96^3 and of the 64^3 coarse mesh + kernels = 2.56 GB on
    the 256^3 workload; 21 B per particle with 16-bit velocities."""
    import bench
    cfg = dict(n_fine=256, coarse_ratio=4, tile=64, buffer=16)
    n = (128 ** 3, 256 ** 3)
    cells = 64 * 96 ** 3 + 64 ** 3
    kernels = 2 * 64 ** 3 + 3 * 4 * 96 * 96 * 49
    assert bench.step_model_bytes(cfg, n, 8) == sum(n) * 15 + 40 * cells + kernels
    assert bench.step_model_bytes(cfg, n, 16) == sum(n) * 21 + 40 * cells + kernels
    assert abs(bench.step_model_bytes(cfg, n, 8) / 1e9 - 2.56) < 0.01
