"""The multi-GPU form is replicas only: every rank runs its own stream (no data-path collective), the
timed region is the slowest rank's, and the reported rate is the units of all ranks over that time.
This exercises the bench's replica logic with two gloo ranks on CPU, each running the CPU oracle on
its own seeded stream."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        from oracle.ttice_oracle import TTICEOracle
        from tt_streams import blob_video

        seed = bench.replica_seed(rank)
        y = blob_video(0, 4, height=24, width=32, n_blobs=3, sigma=(2, 5), view=(4, 6, 4, 8, 3), seed=seed)
        o = TTICEOracle((4, 6, 4, 8, 3), 0.1)
        for k in range(0, 4, 2):
            o.update(y[k:k + 2].double().numpy())
        # a rank-dependent "elapsed time": the slowest is rank ws-1
        elapsed = 1.0 + rank
        slowest = bench.max_over_ranks(elapsed, ws, torch.device("cpu"))
        rate = bench.whole_job_rate(ws, 4 * y[0].numel(), slowest)
        out[rank] = (seed, list(o.ranks), float(np.abs(o.reconstruct(0, 4)).sum()), slowest, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
    (s0, r0, a0, t0, v0), (s1, r1, a1, t1, v1) = out[0], out[1]
    assert s0 != s1                      # independent streams
    assert a0 != a1                      # ... so the replicas hold different representations
    assert t0 == t1 == 2.0               # both ranks report the slowest rank's time
    n = 4 * 4 * 6 * 4 * 8 * 3
    assert v0 == v1 == pytest.approx(ws * n / 2.0)
    assert r0[0] == r1[0] == 1          # r_0 = 1 on both replicas
