"""Splitting a phase scan across ranks (one process per GPU) and merging labels.

Parameter points are independent (Sec. 3: all (q, k, Delta) combinations can be
computed separately), so ranks take disjoint parts of the q list and run the
whole path on their part with no collective in the data path.  Q = 0 stays on
every rank because it defines the normal-state reference Omega_N of every
label.  The only exchange is at the end: per (h, T) point each rank reports its
best superconducting candidate (Omega*, global q index), and the winner over
ranks gives the label -- the outer argmin of Alg. 1 over the union of q.
"""
from __future__ import annotations

import numpy as np

NORMAL, BCS, FFLO = 0, 1, 2


def shard_q(n_q: int, rank: int, world: int, zero_index: int = 0):
    """Global q indices of this rank: q[zero_index] plus every world-th other q."""
    others = [i for i in range(n_q) if i != zero_index]
    return [zero_index] + [i for j, i in enumerate(others) if j % world == rank]


def local_candidates(omega_star, omega_lo, q_global, q_is_zero, tau_rel=1e-12):
    """Per point, the rank's best candidate: (omega_best, q_best_global or -1, omega_N).

    omega_star, omega_lo: [n_q_local, n_pts] from the rank's scan; q_global: the
    global index of each local q; q_is_zero: bool per local q."""
    ws = np.asarray(omega_star, dtype=np.float64)
    w0 = np.asarray(omega_lo, dtype=np.float64)
    qz = np.asarray(q_is_zero, dtype=bool)
    z = int(np.flatnonzero(qz)[0])
    omega_n = w0[z]
    tau = tau_rel * np.abs(omega_n)
    cand = ws < w0 - tau
    masked = np.where(cand, ws, np.inf)
    # lowest Omega, ties to the lowest global q index
    order = np.lexsort((np.asarray(q_global)[:, None].repeat(ws.shape[1], 1), masked), axis=0)
    best_local = order[0]
    cols = np.arange(ws.shape[1])
    best_val = masked[best_local, cols]
    best_q = np.where(np.isfinite(best_val), np.asarray(q_global)[best_local], -1)
    return best_val, best_q, omega_n


def merge_candidates(best_vals, best_qs, omega_n, zero_q: int = 0, tau_rel=1e-12):
    """Labels from the stacked per-rank candidates ([world, n_pts] each)."""
    v = np.asarray(best_vals, dtype=np.float64)
    q = np.asarray(best_qs)
    key_q = np.where(q < 0, np.iinfo(np.int64).max, q)
    order = np.lexsort((key_q, v), axis=0)[0]
    cols = np.arange(v.shape[1])
    vb = v[order, cols]
    qb = q[order, cols]
    tau = tau_rel * np.abs(omega_n)
    win = np.isfinite(vb) & (vb < omega_n - tau)
    labels = np.where(win, np.where(qb == zero_q, BCS, FFLO), NORMAL).astype(np.int8)
    return labels, np.where(win, qb, -1)


def gather_labels(best_val, best_q, omega_n, zero_q: int = 0):
    """All-gather the per-rank candidates with torch.distributed and merge them."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size()
    dev = torch.device("cuda") if dist.get_backend() == "nccl" else torch.device("cpu")
    tv = torch.as_tensor(np.asarray(best_val, dtype=np.float64), device=dev)
    tq = torch.as_tensor(np.asarray(best_q, dtype=np.int64), device=dev)
    vs = [torch.empty_like(tv) for _ in range(world)]
    qs = [torch.empty_like(tq) for _ in range(world)]
    dist.all_gather(vs, tv)
    dist.all_gather(qs, tq)
    return merge_candidates(np.stack([x.cpu().numpy() for x in vs]), np.stack([x.cpu().numpy() for x in qs]),
                            omega_n, zero_q)
