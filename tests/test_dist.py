"""Multi-rank host logic of the replica path, on CPU with the gloo backend (world size 2).

The FDAS path shards by independent spectra (DM trials): each rank searches its own spectrum
and nothing is exchanged on the data path. Only the timing reduction crosses ranks.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        seed = bench.rank_seed(r)
        wl = synth.ska_workload(n=1 << 12, seed=seed)
        slowest = bench.max_over_ranks(1.0 + r, w)  # rank r "took" 1 + r seconds
        out[r] = (w, r, seed, wl.spectrum[:4].tobytes(), slowest, bench.job_throughput(w, 10, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_spectra_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert sorted(res) == [0, 1]
    (w0, r0, s0, b0, t0, v0), (w1, r1, s1, b1, t1, v1) = res[0], res[1]
    assert (w0, w1, r0, r1) == (2, 2, 0, 1)
    assert s0 != s1 and b0 != b1  # distinct spectra per rank
    assert t0 == t1 == 2.0  # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 10 / 2.0)  # whole-job units over the max time
