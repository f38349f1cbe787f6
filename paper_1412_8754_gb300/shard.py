"""Splitting a phase scan across ranks (one process per GPU) and merging labels.

Parameter points are independent (Sec. 3: all (q, k, Delta) combinations can be
computed separately), so ranks take disjoint parts of the q list and run the
whole path on their part with no collective in the data path.  Q = 0 lives on
rank 0 only: it defines the normal-state reference Omega_N of every label, which
rank 0 broadcasts once.  The only exchange is at the end: per (h, T) point each
rank reports its best superconducting candidate (Omega*, global q index), and
the winner over ranks gives the label -- the outer argmin of Alg. 1 over the
union of q.  The candidate and merge rules run in the library
(ffe_label_candidates, ffe_merge_candidates); this module only marshals the
arrays and calls torch.distributed.
"""
from __future__ import annotations


import numpy as np

from . import ffe


def shard_q(n_q: int, rank: int, world: int, zero_index: int = 0):
    """Global q indices of this rank: round robin over the whole list, starting at zero_index on
    rank 0 (so Q = 0 is scanned once, by rank 0)."""
    return [i for i in range(n_q) if (i - zero_index) % world == rank]


def _lib():
    return ffe.lib()


def local_candidates(per_point, q_global, omega_n):
    """Per point, the rank's best candidate: (omega_best [+inf where none], q_best_global or -1).

    per_point: [n_q_local, n_pts] results (ffe.RESULT_DTYPE) of the rank's scan; q_global: the
    global index of each local q; omega_n: [n_pts] normal states Omega(q = 0, Delta = 0)."""
    r = np.ascontiguousarray(per_point, dtype=ffe.RESULT_DTYPE)
    n_q, n_pts = r.shape
    qg = np.ascontiguousarray(q_global, dtype=np.int32)
    on = np.ascontiguousarray(omega_n, dtype=np.float64)
    bv = np.zeros(n_pts)
    bq = np.zeros(n_pts, dtype=np.int32)
    st = _lib().ffe_label_candidates(ffe._ptr(r), n_q, n_pts, ffe._ptr(qg), ffe._ptr(on), ffe._ptr(bv), ffe._ptr(bq))
    if st != ffe.FFE_OK:
        raise ffe.FFEError(st, "ffe_label_candidates")
    return bv, bq


def merge_candidates(best_vals, best_qs, omega_n, zero_q: int = 0):
    """Labels and best q from the stacked per-rank candidates ([world, n_pts] each)."""
    v = np.ascontiguousarray(best_vals, dtype=np.float64)
    q = np.ascontiguousarray(best_qs, dtype=np.int32)
    on = np.ascontiguousarray(omega_n, dtype=np.float64)
    world, n_pts = v.shape
    labels = np.zeros(n_pts, dtype=np.int8)
    best = np.zeros(n_pts, dtype=np.int32)
    st = _lib().ffe_merge_candidates(world, n_pts, ffe._ptr(v), ffe._ptr(q), ffe._ptr(on), int(zero_q),
                                     ffe._ptr(labels), ffe._ptr(best))
    if st != ffe.FFE_OK:
        raise ffe.FFEError(st, "ffe_merge_candidates")
    return labels, best


def _device():
    import torch
    import torch.distributed as dist

    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def broadcast_normal_state(omega_n, src: int = 0):
    """Omega_N [n_pts] from the rank that scanned Q = 0 (src) to every rank."""
    import torch
    import torch.distributed as dist

    t = torch.as_tensor(np.asarray(omega_n, dtype=np.float64), device=_device()).contiguous()
    dist.broadcast(t, src=src)
    return t.cpu().numpy()


def gather_labels(best_val, best_q, omega_n, zero_q: int = 0):
    """All-gather the per-rank candidates with torch.distributed and merge them."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size()
    dev = _device()
    tv = torch.as_tensor(np.asarray(best_val, dtype=np.float64), device=dev)
    tq = torch.as_tensor(np.asarray(best_q, dtype=np.int32), device=dev)
    vs = [torch.empty_like(tv) for _ in range(world)]
    qs = [torch.empty_like(tq) for _ in range(world)]
    dist.all_gather(vs, tv)
    dist.all_gather(qs, tq)
    return merge_candidates(np.stack([x.cpu().numpy() for x in vs]), np.stack([x.cpu().numpy() for x in qs]),
                            omega_n, zero_q)
