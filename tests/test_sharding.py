"""Multi-rank phase scans: q sharding and label merge, world size 2 over gloo on CPU.

The per-q minima come from the FP64 oracle on a small lattice; the labels merged
across two ranks must equal the single-process labels over the whole q list."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from oracle import search
from paper_1412_8754_gb300 import shard

N, U = 16, 4.0
QX = np.array([0.0, 0.1, 0.2, 0.3, 0.45, 0.6, 0.75])
H = np.array([0.0, 0.06, 0.12])
T = np.array([0.004, 0.02])
GRID = np.linspace(0.0, 0.2, 21)


def minima(q_idx):
    """(omega_star, omega_lo) [len(q_idx), n_pts] from the oracle's grid search."""
    m = oracle.make_model(U=U)
    HH, TT = np.meshgrid(H, T, indexing="ij")
    HH, TT = HH.ravel(), TT.ravel()
    ws = np.zeros((len(q_idx), HH.size))
    w0 = np.zeros_like(ws)
    for a, qi in enumerate(q_idx):
        for p in range(HH.size):
            om, _, _ = oracle.omega_batch(m, N, QX[qi], 0.0, HH[p], TT[p], GRID, nthreads=1)
            ws[a, p] = om[search.grid_argmin(om)]
            w0[a, p] = om[0]
    return ws, w0


def test_shard_q_partition():
    for world in (1, 2, 3, 5):
        parts = [shard.shard_q(len(QX), r, world) for r in range(world)]
        others = sorted(i for p in parts for i in p[1:])
        assert others == list(range(1, len(QX)))
        assert all(p[0] == 0 for p in parts)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    q_idx = shard.shard_q(len(QX), rank, world)
    ws, w0 = minima(q_idx)
    bv, bq, omega_n = shard.local_candidates(ws, w0, q_idx, QX[q_idx] == 0.0)
    labels, best = shard.gather_labels(bv, bq, omega_n)
    out[rank] = (labels.tolist(), best.tolist())
    dist.destroy_process_group()


def test_two_rank_labels_equal_single_process():
    ws, w0 = minima(list(range(len(QX))))
    ref = [search.phase_label(ws[:, p], w0[:, p], QX == 0.0) for p in range(ws.shape[1])]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        got = dict(out)
    for rank in range(2):
        labels, best = got[rank]
        assert labels == [r[0] for r in ref]
        assert best == [r[1] for r in ref]
    assert any(r[0] != search.NORMAL for r in ref)  # the case is not trivially normal
