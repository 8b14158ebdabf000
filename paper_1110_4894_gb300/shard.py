"""Host-side logic of a run over several GPUs (one process per GPU).

Bundles are independent lines of sight, so a multi-GPU run splits them
between ranks and needs one exchange at the end: the muPDF.  Every rank
gathers every rank's histogram and the library's rt3d_histogram_combine
rebuilds the histogram of the union (counts and fixed-point weights exactly,
the weighted moments from each rank's weight, mean and spread).  Nothing here
runs on the data path of a trace.
"""
import numpy as np


def shard_range(n, rank, world):
    """contiguous [lo, hi) of n items for rank of world (sizes differ by at most one)"""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d of world %d" % (rank, world))
    q, r = divmod(int(n), world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def combine_histograms(parts):
    """the muPDF of the union of the ranks' bundles from per-rank
    (counts, wfix, scalars), by the library's rt3d_histogram_combine (exact
    for counts and weights; moments from each part's weight, mean and spread)"""
    from ._binding import histogram_combine
    return histogram_combine(parts)


def allreduce_histogram(counts, wfix, sc, group=None, device=None):
    """combine_histograms across a torch.distributed process group: every
    rank gathers every rank's histogram (two integer vectors and eight
    scalars) and combines them with the library (device: where the exchanged
    tensors live, e.g. the rank's GPU for nccl; None = CPU, for gloo)"""
    import torch
    import torch.distributed as dist
    from ._binding import _HIST_KEYS
    world = dist.get_world_size(group)
    c = torch.from_numpy(np.asarray(counts, np.uint64).view(np.int64).copy())
    w = torch.from_numpy(np.asarray(wfix, np.uint64).view(np.int64).copy())
    v = torch.tensor([float(sc[k]) for k in _HIST_KEYS], dtype=torch.float64)
    if device is not None:
        c, w, v = c.to(device), w.to(device), v.to(device)
    gathered = []
    for t in (c, w, v):
        out = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(out, t, group=group)
        gathered.append([o.cpu().numpy() for o in out])
    parts = []
    for r in range(world):
        vals = gathered[2][r]
        scr = {k: (int(vals[i]) if i < 5 else float(vals[i])) for i, k in enumerate(_HIST_KEYS)}
        parts.append((gathered[0][r].view(np.uint64), gathered[1][r].view(np.uint64), scr))
    return combine_histograms(parts)


def rank_lines_of_sight(theta, rank):
    """a rank's own bundle centres for a weak-scaling run: the grid moved by
    half its spacing for ranks 4-7, then turned by rank x 90 degrees about
    the optical axis, so that each of up to eight ranks traces different
    lines of sight"""
    t = np.asarray(theta, np.float64).copy()
    if (rank // 4) % 2:
        xs = np.unique(t[:, 0])
        step = float(np.min(np.diff(xs))) if xs.size > 1 else 0.0
        t += 0.5 * step
    for _ in range(rank % 4):
        t = np.stack([-t[:, 1], t[:, 0]], axis=1)
    return np.ascontiguousarray(t)
