"""The multi-GPU host logic on the CPU: bundles split between ranks, the
muPDF combined across two gloo ranks equals the muPDF of all bundles
(integer counts and weights exactly, moments to rounding)."""
import os
import socket

import numpy as np
import pytest

import inputs
import oracle
from paper_1110_4894_gb300.shard import allreduce_histogram, combine_histograms, shard_range


def test_shard_range_covers_everything_once():
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            spans = [shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _mu(n=5000, seed=19):
    g = inputs.rng(seed)
    mu = np.exp(g.uniform(np.log(0.6), np.log(4.0), n))
    mu[::17] *= -1
    flags = np.zeros(n, np.int32)
    flags[::131] = oracle.F_NOCROSS
    return mu, flags


def _check(got, want):
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    for k in ("n_used", "n_under", "n_over", "n_neg", "n_bad"):
        assert got[2][k] == want[2][k]
    for k in ("W_total", "mean_w", "sigma_w"):
        assert abs(got[2][k] / want[2][k] - 1) < 1e-12


def test_combine_histograms_equals_the_whole():
    mu, flags = _mu()
    whole = oracle.histogram(mu, flags, 120, 0.5, 5.0)
    parts = []
    for r in range(3):
        lo, hi = shard_range(len(mu), r, 3)
        parts.append(oracle.histogram(mu[lo:hi], flags[lo:hi], 120, 0.5, 5.0))
    _check(combine_histograms(parts), whole)


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mu, flags = _mu()
        lo, hi = shard_range(len(mu), rank, world)
        c, w, sc = oracle.histogram(mu[lo:hi], flags[lo:hi], 120, 0.5, 5.0)
        q.put((rank, allreduce_histogram(c, w, sc)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_mupdf():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mu, flags = _mu()
    whole = oracle.histogram(mu, flags, 120, 0.5, 5.0)
    _check(out[0], whole)
    _check(out[1], whole)


def test_ranks_trace_different_lines_of_sight():
    from paper_1110_4894_gb300.shard import rank_lines_of_sight
    th = inputs.config_c2(n_particles=10, n_side=8, n_steps=10)["theta"]
    sets = [set(map(tuple, np.round(rank_lines_of_sight(th, r) * 1e9).astype(np.int64))) for r in range(8)]
    for a in range(8):
        assert len(sets[a]) == len(th)
        for b in range(a):
            assert not (sets[a] & sets[b])


def test_combine_shear_histograms_equals_the_whole():
    # the shear PDF's weighted mean is not n_used / W: the combination must
    # use each part's own mean and spread
    g = inputs.rng(23)
    n = 4000
    gam = np.exp(g.uniform(np.log(1e-3), np.log(0.5), n))
    ang = g.uniform(0, 2 * np.pi, n)
    g1, g2 = gam * np.cos(ang), gam * np.sin(ang)
    mu = np.exp(g.uniform(np.log(0.5), np.log(5.0), n))
    flags = np.zeros(n, np.int32)
    whole = oracle.shear_histogram(mu, g1, g2, flags, 64, 1e-3, 1.0)
    parts = []
    for r in range(4):
        lo, hi = shard_range(n, r, 4)
        parts.append(oracle.shear_histogram(mu[lo:hi], g1[lo:hi], g2[lo:hi], flags[lo:hi], 64, 1e-3, 1.0))
    _check(combine_histograms(parts), whole)


def test_combine_rejects_bad_parts():
    import paper_1110_4894_gb300 as P
    mu, flags = _mu(200)
    c, w, sc = oracle.histogram(mu, flags, 10, 0.5, 5.0)
    bad = dict(sc, W_total=-1.0)
    with pytest.raises(P.Rt3dError):
        combine_histograms([(c, w, sc), (c, w, bad)])
    with pytest.raises(ValueError):
        combine_histograms([(c, w, sc), (c[:5], w[:5], sc)])
