"""The multi-rank (data-parallel) path on CPU: world_size 2, gloo backend.

Each rank owns a shard of the batch (`distributed.shard`). The forward and
data gradient of a shard need nothing from the other rank; the weight and
bias gradients are sums over the batch, so the per-shard partial sums added
over the ranks (`distributed.all_reduce_sum_`) must equal the gradient of the
whole batch. The per-shard gradients here come from the FP64 oracle (this is
test code), so the check is the partition logic and the one exchange, not
the GPU kernels.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2207_00257_gb300 import distributed as D


def test_shard_partitions_the_batch():
    for n_total in (0, 1, 5, 6, 32, 33):
        for world in (1, 2, 3, 4, 8):
            spans = [D.shard(n_total, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n_total
            for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
                assert a1 == b0  # contiguous, in rank order
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.shard(4, 2, 2)
    with pytest.raises(ValueError):
        D.shard(4, 0, 0)


def test_weak_scaling_rate():
    assert D.weak_scaling_rate(10.0, 4, 2.0) == 20.0
    with pytest.raises(ValueError):
        D.weak_scaling_rate(1.0, 1, 0.0)


def test_single_process_helpers_without_a_group():
    assert D.max_over_ranks(3.5) == 3.5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2207_00257_gb300.synth import ConvShape, make_inputs

        # a small strided layer, NHWC, batch 5 split 3 + 2
        sh = ConvShape(5, 4, 7, 6, 3, 3, 3, 2, 1, 1, layout="NHWC")
        x, w, b, g = make_inputs(sh, seed=11, grad=True)
        n0, n1 = D.shard(sh.N, rank, world)
        full = oracle.Conv(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, 2, 1, 1, "NHWC")
        part = oracle.Conv(n1 - n0, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, 2, 1, 1, "NHWC")
        xs, gs = x[n0:n1].double().numpy(), g[n0:n1].double().numpy()
        dw = torch.from_numpy(oracle.conv2d_wgrad(part, xs, gs).copy())
        db = torch.from_numpy(oracle.conv2d_bgrad(part, gs).copy())
        D.all_reduce_sum_([dw, db])
        # the timing reduction: the job is as slow as its slowest rank
        slowest = D.max_over_ranks(1.0 + rank, device="cpu")
        if rank == 0:
            dw_ref = oracle.conv2d_wgrad(full, x.double().numpy(), g.double().numpy())
            db_ref = oracle.conv2d_bgrad(full, g.double().numpy())
            err_w = float(np.max(np.abs(dw.numpy() - dw_ref)) / max(np.max(np.abs(dw_ref)), 1e-300))
            err_b = float(np.max(np.abs(db.numpy() - db_ref)) / max(np.max(np.abs(db_ref)), 1e-300))
            with open(result_path, "w") as f:
                f.write(f"{err_w} {err_b} {slowest}\n")
    finally:
        dist.destroy_process_group()


def test_data_parallel_weight_gradient_gloo(tmp_path):
    world = 2
    out = tmp_path / "result.txt"
    mp.start_processes(_worker, args=(world, _free_port(), str(out)), nprocs=world, join=True,
                       start_method="spawn")
    err_w, err_b, slowest = (float(v) for v in out.read_text().split())
    # the sum over shards equals the full-batch sum up to FP64 reassociation
    assert err_w < 1e-13 and err_b < 1e-13
    assert slowest == 2.0
