"""Multi-rank phase scans: q sharding and label merge, world size 2 over gloo on CPU.

The per-q minima come from the FP64 oracle on a small lattice; the labels merged
across ranks (the library's host functions ffe_label_candidates and
ffe_merge_candidates) must equal the single-process labels over the whole q list."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from oracle import search
from paper_1412_8754_gb300 import ffe, shard

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
        assert sorted(i for p in parts for i in p) == list(range(len(QX)))  # each q once
        assert 0 in parts[0]  # Q = 0 on rank 0 only
        assert max(map(len, parts)) - min(map(len, parts)) <= 1


def results(ws, w0):
    r = np.zeros(ws.shape, dtype=ffe.RESULT_DTYPE)
    r["omega_star"], r["omega_lo"] = ws, w0
    return r


def test_merge_rules_match_the_single_process_labels():
    """The library's candidate and merge rules (host code, no GPU) give, for every split of the q
    list, the labels the oracle's phase_label gives over the whole list."""
    ws, w0 = minima(list(range(len(QX))))
    ref = [search.phase_label(ws[:, p], w0[:, p], QX == 0.0) for p in range(ws.shape[1])]
    omega_n = w0[0]
    for world in (1, 2, 3, 7):
        cands = [shard.local_candidates(results(ws[q], w0[q]), q, omega_n)
                 for q in (shard.shard_q(len(QX), r, world) for r in range(world))]
        labels, best = shard.merge_candidates([c[0] for c in cands], [c[1] for c in cands], omega_n)
        assert labels.tolist() == [r[0] for r in ref] and best.tolist() == [r[1] for r in ref], world
    # ties go to the lowest global q index, across ranks as within one
    v = np.array([[-5.0, np.inf], [-5.0, -1.0]])
    q = np.array([[3, -1], [2, 4]], dtype=np.int32)
    labels, best = shard.merge_candidates(v, q, np.array([-1.0, -1.0]))
    assert best.tolist() == [2, -1] and labels.tolist() == [search.FFLO, search.NORMAL]


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
    # rank 0 scanned Q = 0 (its first line): the normal states go to every rank
    omega_n = shard.broadcast_normal_state(w0[0] if rank == 0 else np.zeros(w0.shape[1]), src=0)
    bv, bq = shard.local_candidates(results(ws, w0), q_idx, omega_n)
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
