"""Host logic of multi-GPU runs (one process per GPU, torch.distributed).

The batched domains are independent (each has its own time step), so several
GPUs share no data while they step: a run either gives every rank its own
batch (weak scaling) or splits one batch by longest-processing-time balancing
of the cell counts (strong scaling).  The only collectives are after the timed
region: the maximum of the ranks' times and the sum of their cell-updates.
"""
import heapq

import numpy as np


def lpt_partition(n_cells, world):
    """Domain indices per rank: the longest domains first, each to the rank
    with the fewest cells so far.  Returns a list of sorted index arrays."""
    n_cells = np.asarray(n_cells, dtype=np.int64)
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for d in np.argsort(-n_cells, kind="stable"):
        load, r = heapq.heappop(heap)
        parts[r].append(int(d))
        heapq.heappush(heap, (load + int(n_cells[d]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def reduce_time_and_work(ms, updates, device=None):
    """(max of ms over ranks, sum of updates over ranks); identity without an
    initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(updates)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
