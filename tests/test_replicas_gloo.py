"""Host-side logic of the multi-GPU replica benchmark, on CPU with gloo.

Each rank runs its own plan on its own channels; the only communication is
the barrier and the max (time) / sum (samples) over ranks.  Two CPU ranks check
that aggregation, that a rank's seed is distinct, and that the launcher
environment is read the way torchrun sets it."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        t = bench.max_over_ranks(10.0 + rank, world)             # per-rank timed region (ms)
        n = bench.sum_over_ranks(1000.0 * (rank + 1), world)      # per-rank samples
        bench.barrier(world)
        queue.put((rank, w, r, local, t, n))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, w, r, local, t, n in res:
        assert (w, r, local) == (2, rank, rank)
        assert t == 11.0                 # max over ranks
        assert n == 3000.0               # sum over ranks


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.sum_over_ranks(7.0, 1) == 7.0
    bench.barrier(1)


def test_channel_subset_workload_keeps_geometry():
    """The profiling subset keeps the channel width, N, overlap and hop."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle as O
    w_full, q_full = bench.workload_info()
    w_sub, q_sub = bench.workload_info(128)
    assert q_full == q_sub == 76
    assert w_sub.chan_bw_mhz == pytest.approx(w_full.chan_bw_mhz)
    g_full = O.plan_geometry(w_full.f_center_mhz, w_full.bandwidth_mhz, w_full.n_chan, w_full.dm,
                             w_full.n_fft, w_full.n_avg)
    g_sub = O.plan_geometry(w_sub.f_center_mhz, w_sub.bandwidth_mhz, w_sub.n_chan, w_sub.dm,
                            w_sub.n_fft, w_sub.n_avg)
    assert (g_full.n_ov, g_full.hop) == (g_sub.n_ov, g_sub.hop) == (64, 8128)
    assert list(g_sub.shift) == list(g_full.shift[:128])
