"""rt3d_potential_device_noalloc against rt3d_potential.

The no-allocation entry point serves callers that cannot call cudaMalloc
(device memory already reserved in full by another framework's pool, or code
that must not pay the synchronisation an allocation can imply).  It runs the
same pair-sum kernels with the split partials in a static device array, so its
output must agree with rt3d_potential within the pair-sum tolerances; two
calls in a row check that the shared array's leftovers never leak into a
result.  This file is collected last on purpose."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def _compare(out, ref, fp64):
    e_phi = np.abs(out[:, 0] - ref[:, 0]) / np.abs(ref[:, 0])
    e_g = np.linalg.norm(out[:, 1:] - ref[:, 1:], axis=1) / np.linalg.norm(ref[:, 1:], axis=1)
    if fp64:
        assert e_phi.max() < 1e-12 and e_g.max() < 1e-11
    else:
        assert e_phi.max() < 2e-6
        assert np.percentile(e_g, 99) < 5e-6 and e_g.max() < 5e-5


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_potential_isolated(precision):
    import torch

    import paper_1110_4894_gb300 as P
    ctx = P.Context(0, precision=precision)
    ctx.set_cosmology()
    g = inputs.rng(123)
    n = 3 * 256 + 41
    pos = inputs.quantize(np.array([0.0, 0.0, 900.0]) + g.normal(size=(n, 3)) * 0.5)
    ctx.load_particles(4, pos, g.uniform(0.5, 2.0, n) * 1e10, 0.01)
    stream = torch.cuda.current_stream()
    for call in range(2):
        m = 700 + 300 * call
        pts = np.array([0.0, 0.0, 900.0]) + g.normal(size=(m, 3)) * (0.6 + call)
        ref = ctx.potential(4, pts)
        d_pts = torch.from_numpy(np.ascontiguousarray(pts.T)).cuda()
        d_out = torch.full((m * 4,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.potential_device_noalloc(stream.cuda_stream, 4, m, d_pts.data_ptr(), 0, d_out.data_ptr())
        torch.cuda.synchronize()
        _compare(d_out.cpu().numpy().reshape(m, 4), ref, precision == 1)
    ctx.close()


def test_noalloc_matches_potential_replicated():
    import torch

    import paper_1110_4894_gb300 as P
    ctx = P.Context(0)
    ctx.set_cosmology()
    L = inputs.box_length(20.0 / 0.7)
    pos, mass, _ = inputs.halo_box(3000, L, 8, seed=77)
    rot, shift = inputs.replicas(4, L, seed=77)
    ctx.load_particles(2, pos, mass, 0.02, replicated=True, box_length=L, rot=rot, shift=shift, mean_subtract=True)
    g = inputs.rng(9)
    stream = torch.cuda.current_stream()
    for call in range(2):
        m = 500 + 211 * call
        rep = g.integers(0, 4, m).astype(np.int32)
        pts = np.stack([g.uniform(-0.5, 0.5, m) * L, g.uniform(-0.5, 0.5, m) * L, (rep + g.random(m)) * L], 1)
        ref = ctx.potential(2, pts, rep)
        d_pts = torch.from_numpy(np.ascontiguousarray(pts.T)).cuda()
        d_rep = torch.from_numpy(rep).cuda()
        d_out = torch.full((m * 4,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.potential_device_noalloc(stream.cuda_stream, 2, m, d_pts.data_ptr(), d_rep.data_ptr(),
                                     d_out.data_ptr())
        torch.cuda.synchronize()
        out = d_out.cpu().numpy().reshape(m, 4)
        # mean subtraction leaves a small net field: compare against the raw scale
        sc = np.linalg.norm(ref[:, 1:], axis=1).max()
        assert np.all(np.abs(out[:, 1:] - ref[:, 1:]) < 1e-5 * sc)
        assert np.all(np.abs(out[:, 0] - ref[:, 0]) < 1e-6 * np.abs(ref[:, 0]).max())
    with pytest.raises(P.Rt3dError) as e:
        ctx.potential_device_noalloc(stream.cuda_stream, 2, (32 << 20) // 32 + 1, d_pts.data_ptr(), 0,
                                     d_out.data_ptr())
    assert e.value.code == -1
    ctx.close()


def test_noalloc_bad_points_give_nan_and_spare_the_rest():
    """Replica indices outside [0, n_replicas) and non-finite points arrive
    in device memory, where the host cannot check them: the kernels skip them
    and write NaN for exactly those points; every other point, including the
    ones that share a block with a bad first point, keeps its value."""
    import torch

    import paper_1110_4894_gb300 as P
    ctx = P.Context(0)
    ctx.set_cosmology()
    L = inputs.box_length(20.0 / 0.7)
    pos, mass, _ = inputs.halo_box(3000, L, 8, seed=78)
    rot, shift = inputs.replicas(4, L, seed=78)
    ctx.load_particles(3, pos, mass, 0.02, replicated=True, box_length=L, rot=rot, shift=shift, mean_subtract=True)
    g = inputs.rng(10)
    m = 600
    rep = np.sort(g.integers(0, 4, m)).astype(np.int32)
    pts = np.stack([g.uniform(-0.5, 0.5, m) * L, g.uniform(-0.5, 0.5, m) * L, (rep + g.random(m)) * L], 1)
    ref = ctx.potential(3, pts, rep)
    bad_rep = {5: -1, 300: 4, 301: 1 << 30}
    bad_pt = [0, 450]  # index 0 is the anchor of the first block of points
    rep_d, pts_d = rep.copy(), pts.copy()
    for i, r in bad_rep.items():
        rep_d[i] = r
    pts_d[0, 1] = np.nan
    pts_d[450, 2] = np.inf
    stream = torch.cuda.current_stream()
    d_pts = torch.from_numpy(np.ascontiguousarray(pts_d.T)).cuda()
    d_rep = torch.from_numpy(rep_d).cuda()
    d_out = torch.zeros((m * 4,), dtype=torch.float64, device="cuda")
    ctx.potential_device_noalloc(stream.cuda_stream, 3, m, d_pts.data_ptr(), d_rep.data_ptr(), d_out.data_ptr())
    torch.cuda.synchronize()
    out = d_out.cpu().numpy().reshape(m, 4)
    bad = sorted(list(bad_rep) + bad_pt)
    assert np.all(np.isnan(out[bad]))
    good = np.setdiff1d(np.arange(m), bad)
    assert np.all(np.isfinite(out[good]))
    sc = np.linalg.norm(ref[:, 1:], axis=1).max()
    # the first block lost its anchor and measures offsets from the replica
    # frame's origin instead (FP32 rounding of ~L): a looser bound there
    assert np.all(np.abs(out[good, 1:] - ref[good, 1:]) < 1e-3 * sc)
    far = good[good >= 256]
    assert np.all(np.abs(out[far, 1:] - ref[far, 1:]) < 1e-5 * sc)
    ctx.close()
