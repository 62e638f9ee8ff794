"""Multi-rank sharding on CPU (gloo, world size 2): each rank takes its
contiguous template range, computes 2F with the FP64 oracle (standing in for
its GPU), and the gathered result equals a single-process run bit for bit."""
import os
import socket

import numpy as np
import pytest

import synth
from paper_0912_4255_gb300.shard import shard, shard_ranges


def test_ranges_cover_and_balance():
    rng = synth.rng(1)
    nf = 2 ** rng.integers(18, 22, 300)
    for world in (1, 2, 3, 8):
        r = shard_ranges(nf, world)
        assert r[0][0] == 0 and r[-1][1] == len(nf)
        assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))
        w = [float(np.sum(nf[s:e] * np.log2(nf[s:e]))) for s, e in r]
        assert max(w) - min(w) <= 2 * float(np.max(nf) * np.log2(np.max(nf)))
    assert shard_ranges(np.full(8192, 1 << 22), 4) == [(0, 2048), (2048, 4096), (4096, 6144), (6144, 8192)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import fstat as F
    desc = synth.PlanDesc(dt=0.5, n_data=3000, n_fft=4096, interp=1, max_templates=8)
    x = synth.complex_noise(desc.n_data, 1.0, 3)
    a, d = synth.fibonacci_sky(6)
    tm = synth.make_templates(a, d, 0.0, 0, desc.n_data)
    mine, (s, e) = shard(tm, rank, world)
    local = [F.resample_two_f(x.astype(np.complex128), t, np.zeros((0, 2), np.int64), desc) for t in mine]
    gathered = [None] * world
    dist.all_gather_object(gathered, (s, e, local))
    if rank == 0:
        full = np.stack([v for part in sorted(gathered, key=lambda g: g[0]) for v in part[2]])
        ref = np.stack([F.resample_two_f(x.astype(np.complex128), t, np.zeros((0, 2), np.int64), desc)
                        for t in tm])
        np.save(out_path, np.array([np.array_equal(full, ref)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_merge_equals_single_run(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "ok.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert bool(np.load(out)[0])
