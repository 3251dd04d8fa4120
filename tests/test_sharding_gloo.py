"""The multi-GPU design of the matvec (points split across ranks; each rank spreads its points
onto the full grids of every window; one all-reduce (sum) of the grids; each rank runs the FFT
and scaling and interpolates its own points) on CPU ranks over gloo, with the oracle's NFFT
stages standing in for the kernels. Linearity of the spread in v and in the point set makes the
sharded result equal to the unsharded one; the test checks that the exchange sits in the right
place and that every point is interpolated exactly once."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import nfft as on
from synth import minmax_scale

N, M = 16, 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data():
    rng = np.random.default_rng(31)
    X = minmax_scale(rng.standard_normal((240, 6)))
    W = np.array([[0, 1, 2], [3, 4, -1], [5, -1, -1]])
    v = rng.standard_normal(240)
    return X, W, v


def _rank_main(rank, world, port, sizes, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, W, v = _data()
        bounds = np.concatenate([[0], np.cumsum(sizes)])
        lo, hi = bounds[rank], bounds[rank + 1]
        n_os = 2 * N
        beta = on.kb_beta()
        D1 = on.deconv_diag_1d(0.7, N, M, n_os, beta)
        f = np.zeros(hi - lo)
        for win in W:
            feats = [k for k in win if k >= 0]
            xw = X[lo:hi][:, feats]
            g = torch.from_numpy(on.spread_grid(xw, v[lo:hi], n_os, M, beta))
            dist.all_reduce(g, op=dist.ReduceOp.SUM)  # the one exchange per window and matvec
            f += on.interp_grid(xw, on.conv_grid(g.numpy(), D1), n_os, M, beta)
        # collect the shards' results (padded to the largest shard) for the check on rank 0
        pad = max(sizes)
        buf = torch.zeros(pad, dtype=torch.float64)
        buf[: hi - lo] = torch.from_numpy(f)
        bufs = [torch.zeros(pad, dtype=torch.float64) for _ in sizes]
        dist.all_gather(bufs, buf)
        parts = [b[:s] for b, s in zip(bufs, sizes)]
        if rank == 0:
            np.save(out_path, torch.cat(parts).numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("sizes", [[120, 120], [1, 239], [80, 80, 80]])
def test_sharded_matvec_equals_unsharded(tmp_path, sizes):
    X, W, v = _data()
    out_path = str(tmp_path / "kv.npy")
    mp.start_processes(_rank_main, args=(len(sizes), _free_port(), sizes, out_path),
                       nprocs=len(sizes), join=True, start_method="spawn")
    got = np.load(out_path)
    ref = on.nfft_fastsum(X, W, 0.7, N, M, v)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_a_misplaced_exchange_is_caught():
    """Without the all-reduce (each rank interpolating only its own points' grid) the result is
    wrong: the check above is sensitive to the exchange."""
    X, W, v = _data()
    n_os, beta = 2 * N, on.kb_beta()
    D1 = on.deconv_diag_1d(0.7, N, M, n_os, beta)
    halves = [(0, 120), (120, 240)]
    got = np.zeros(240)
    for lo, hi in halves:
        for win in W:
            feats = [k for k in win if k >= 0]
            xw = X[lo:hi][:, feats]
            g = on.spread_grid(xw, v[lo:hi], n_os, M, beta)
            got[lo:hi] += on.interp_grid(xw, on.conv_grid(g, D1), n_os, M, beta)
    ref = on.nfft_fastsum(X, W, 0.7, N, M, v)
    assert np.max(np.abs(got - ref)) > 1e-3 * np.max(np.abs(ref))
