"""The seeded input generators: determinism, the exact position grid, replica
transforms and the NFW sampler's enclosed-mass profile."""
import math

import numpy as np

import inputs


def test_streams_are_deterministic():
    a = inputs.rng(5, 1, 2).random(4)
    b = inputs.rng(5, 1, 2).random(4)
    c = inputs.rng(5, 1, 3).random(4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_box_positions_on_grid_and_inside():
    L = inputs.box_length(20.0)
    pos, mass, info = inputs.halo_box(20000, L, 30, seed=9)
    assert pos.shape == (20000, 3) and np.all(mass == mass[0])
    assert np.all(pos >= 0) and np.all(pos < L)
    k = pos / inputs.QUANTUM
    assert np.array_equal(k, np.round(k))
    assert (L / (2 * inputs.QUANTUM)) == round(L / (2 * inputs.QUANTUM))
    assert info["halo_counts"].sum() == 20000 - info["n_bg"]


def test_replicas_are_proper_rotations():
    R = inputs.proper_rotations()
    assert len(R) == 24
    assert len({r.tobytes() for r in R}) == 24
    for r in R:
        assert np.array_equal(r @ r.T, np.eye(3, dtype=np.int32))
        assert round(np.linalg.det(r)) == 1
    L = inputs.box_length(10.0)
    rot, shift = inputs.replicas(40, L, seed=3)
    assert rot.shape == (40, 3, 3) and np.all(shift >= 0) and np.all(shift < L)
    assert np.array_equal(shift / inputs.QUANTUM, np.round(shift / inputs.QUANTUM))


def test_nfw_sampler_enclosed_mass():
    pos, mass, info = inputs.nfw_halo(1e14, 5.0, 0.25, 1000.0, 200000, seed=1)
    r = np.linalg.norm(pos - np.array([0, 0, 1000.0]), axis=1) / (1.25 * info["rs_phys"])
    m = lambda x: math.log1p(x) - x / (1 + x)
    for x in (0.5, 1.0, 3.0):
        frac = np.mean(r < x)
        assert abs(frac - m(x) / m(10.0)) < 4 * math.sqrt(frac * (1 - frac) / len(r)) + 1e-4
    assert r.max() <= 10.0 + 1e-6
    assert abs(mass.sum() / info["M_trunc"] - 1) < 1e-12


def test_bundle_grid_tiles():
    th = inputs.bundle_grid(-1.0, 1.0, 16, tile=8)
    assert th.shape == (256, 2)
    assert len({tuple(t) for t in th}) == 256
    first = th[:64]
    assert first[:, 0].max() - first[:, 0].min() < 1.0
