"""Host-side logic of a run over several GPUs (one process per GPU).

Bundles are independent lines of sight, so a multi-GPU run splits them
between ranks and needs one exchange at the end: the muPDF.  Counts and
fixed-point weights add exactly (integers); the weighted moments are
recombined from each rank's (n_used, W, mean_w, sigma_w): with w = 1/|mu|,
sum w |mu| = n_used and sum w |mu|^2 = sum |mu| = sigma^2 W + 2 mean n - mean^2 W.
Nothing here runs on the data path of a trace.
"""
import numpy as np


def shard_range(n, rank, world):
    """contiguous [lo, hi) of n items for rank of world (sizes differ by at most one)"""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d of world %d" % (rank, world))
    q, r = divmod(int(n), world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def _moment_sums(sc):
    n, W, m, s = sc["n_used"], sc["W_total"], sc["mean_w"], sc["sigma_w"]
    return np.array([n, sc["n_under"], sc["n_over"], sc["n_neg"], sc["n_bad"], W,
                     s * s * W + 2.0 * m * n - m * m * W], np.float64)


def _from_sums(v):
    n, W, S2 = v[0], v[5], v[6]
    mean = n / W if W > 0 else 0.0
    var = (S2 - 2.0 * mean * n + mean * mean * W) / W if W > 0 else 0.0
    return dict(n_used=int(v[0]), n_under=int(v[1]), n_over=int(v[2]), n_neg=int(v[3]), n_bad=int(v[4]),
                W_total=W, mean_w=mean, sigma_w=float(np.sqrt(max(var, 0.0))))


def combine_histograms(parts):
    """the muPDF of the union of the ranks' bundles from per-rank
    (counts, wfix, scalars); exact for counts and weights"""
    counts = sum(np.asarray(c, np.uint64) for c, _, _ in parts)
    wfix = sum(np.asarray(w, np.uint64) for _, w, _ in parts)
    return counts, wfix, _from_sums(sum(_moment_sums(sc) for _, _, sc in parts))


def allreduce_histogram(counts, wfix, sc, group=None, device=None):
    """combine_histograms across a torch.distributed process group: two
    integer sums and one FP64 sum (device: where the tensors live, e.g. the
    rank's GPU for nccl; None = CPU, for gloo)"""
    import torch
    import torch.distributed as dist
    ts = [torch.from_numpy(np.asarray(counts, np.int64).copy()),
          torch.from_numpy(np.asarray(wfix, np.uint64).view(np.int64).copy()),
          torch.from_numpy(_moment_sums(sc))]
    if device is not None:
        ts = [t.to(device) for t in ts]
    for t in ts:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    c, w, m = (t.cpu().numpy() for t in ts)
    return c.astype(np.uint64), w.view(np.uint64), _from_sums(m)


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
