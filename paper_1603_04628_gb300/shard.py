"""Sharding a batch of micro-elements over ranks (one GPU per rank).

Micro-elements are independent (the paper's quasi-steady subdomains, Sec. 2.1),
so a batch splits into per-rank sub-batches with no exchange during MD.  The
split balances work (atoms x steps) greedily, largest element first (LPT);
the only collective is the gather of the per-element results (a few dozen
bytes each) back to rank 0, in the batch's original order.
"""
import numpy as np


def element_work(el):
    """Atoms x steps of one element (fluid count from the element's density
    and box; walls ~ 12 atoms per wall lattice cell of a0 = 4^(1/3))."""
    nf = round(el["density"] * el["Lx"] * el["h"] * el["Lz"])
    a0 = 4.0 ** (1.0 / 3.0)
    nw = 12 * max(1, round(el["Lx"] / a0)) * max(1, round(el["Lz"] / a0))
    return (nf + nw) * (int(el.get("steps_eq", 0)) + int(el.get("steps_sample", 0)))


def partition(elements, world):
    """Indices of the elements each rank runs: longest work first, each to the
    currently least-loaded rank.  Every element appears exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    work = [element_work(e) for e in elements]
    order = sorted(range(len(elements)), key=lambda i: (-work[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += work[i]
    return [sorted(p) for p in parts]


RESULT_KEYS = ("q", "q_se", "p", "p_se", "T_meas", "e_drift", "n_fluid", "n_wall", "status")


def gather_results(local_results, local_indices, n_total, dist, group=None):
    """Gather every rank's results to rank 0 in the original element order.
    Returns the full list on rank 0 and None elsewhere."""
    import torch
    rows = np.array([[r[k] for k in RESULT_KEYS] for r in local_results], dtype=np.float64).reshape(-1, len(RESULT_KEYS))
    idx = np.asarray(local_indices, dtype=np.float64).reshape(-1, 1)
    payload = torch.from_numpy(np.hstack([idx, rows]))
    world = dist.get_world_size(group)
    # pad to the largest shard so every rank sends the same shape
    n_local = torch.tensor([payload.shape[0]], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n_local, group=group)
    m = int(max(s.item() for s in sizes))
    padded = torch.full((m, payload.shape[1]), -1.0, dtype=torch.float64)
    padded[: payload.shape[0]] = payload
    bufs = [torch.empty_like(padded) for _ in range(world)] if dist.get_rank(group) == 0 else None
    dist.gather(padded, bufs, dst=0, group=group)
    if dist.get_rank(group) != 0:
        return None
    out = [None] * n_total
    for r, buf in enumerate(bufs):
        for row in buf[: int(sizes[r].item())].numpy():
            i = int(row[0])
            d = dict(zip(RESULT_KEYS, row[1:]))
            for k in ("n_fluid", "n_wall", "status"):
                d[k] = int(d[k])
            out[i] = d
    return out
