"""GPU parity of the projectors against the FP64 oracle, through the C ABI.

Tolerances (from the arithmetic: FP32 sample positions carry ~1e-4 voxel of
error at DSO/d ~ 1000-2000 and FP32 sums of ~1000 terms ~1e-6 relative):
relative L2 <= 1e-5 per projection and per volume, max-abs <= 1e-4 of the
reference maximum."""
import numpy as np
import pytest

import oracle
from conftest import max_rel, rel_l2
from paper_2412_10129_gb300 import inputs, tg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_L2 = 1e-5
RTOL_MAX = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_10129_gb300 import build
    build.build()
    tg.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def assert_proj_close(got, ref):
    assert rel_l2(got, ref) <= RTOL_L2, rel_l2(got, ref)
    assert max_rel(got, ref) <= RTOL_MAX, max_rel(got, ref)
    norms = np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)
    for a in np.nonzero(norms > 1e-3 * norms.max())[0]:
        assert rel_l2(got[a], ref[a]) <= RTOL_L2, (a, rel_l2(got[a], ref[a]))


def assert_vol_close(got, ref):
    assert rel_l2(got, ref) <= RTOL_L2, rel_l2(got, ref)
    assert max_rel(got, ref) <= RTOL_MAX, max_rel(got, ref)


@pytest.fixture(scope="module")
def small():
    g = inputs.config_small()
    x = inputs.ellipsoid_phantom(g, 10, seed=1)
    y = inputs.random_projections(g, seed=2)
    return g, x, y


def ragged_geometry(seed=3):
    return inputs.random_geometry((37, 29, 23), (1.0, 1.2, 0.9), (45, 31), (1.3, 1.1), 13, seed=seed,
                                  DSO=300.0, DSD=520.0)


@pytest.mark.parametrize("method", ["interp", "siddon"])
def test_forward_small_workload(small, method):
    g, x, _ = small
    got = host(tg.forward(g, dev(x), method))
    ref = oracle.forward(g, x, method)
    assert_proj_close(got, ref)


@pytest.mark.parametrize("method", ["interp", "siddon"])
def test_forward_ragged_arbitrary_geometry(method):
    g = ragged_geometry()
    x = inputs.random_volume(g, seed=4)
    got = host(tg.forward(g, dev(x), method))
    assert_proj_close(got, oracle.forward(g, x, method))


def test_matched_backprojection_small_workload(small):
    g, _, y = small
    got = host(tg.backproject(g, dev(y), "matched"))
    assert_vol_close(got, oracle.backproject(g, y, "matched"))


def test_matched_backprojection_ragged():
    g = ragged_geometry(5)
    y = inputs.random_projections(g, seed=6)
    got = host(tg.backproject(g, dev(y), "matched"))
    assert_vol_close(got, oracle.backproject(g, y, "matched"))


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_adjoint_identity_on_gpu(small, case):
    if case == "small":
        g = small[0]
    else:
        g = ragged_geometry(8)
    x = dev(inputs.random_volume(g, seed=9))
    y = dev(inputs.random_projections(g, seed=10))
    Ax = tg.forward(g, x, "interp")
    Aty = tg.backproject(g, y, "matched")
    lhs = float(torch.sum(Ax.double() * y.double()))
    rhs = float(torch.sum(x.double() * Aty.double()))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_fdk_weighted_backprojection_ragged():
    g = ragged_geometry(11)
    y = inputs.random_projections(g, seed=12)
    got = host(tg.backproject(g, dev(y), "fdk"))
    assert_vol_close(got, oracle.backproject(g, y, "fdk"))


def test_fdk_small_workload(small):
    g, x, _ = small
    b = oracle.forward(g, x, "siddon").astype(np.float32)  # measured data: any projections
    got = host(tg.fdk(g, dev(b)))
    assert_vol_close(got, oracle.fdk(g, b))


def test_batch_equals_single_calls():
    g = ragged_geometry(13)
    xs = np.stack([inputs.random_volume(g, seed=s) for s in (20, 21, 22)])
    ys = np.stack([inputs.random_projections(g, seed=s) for s in (23, 24, 25)])
    for method in ("interp", "siddon"):
        pb = host(tg.forward(g, dev(xs), method))
        for i in range(3):
            np.testing.assert_array_equal(pb[i], host(tg.forward(g, dev(xs[i]), method)))
    for method in ("matched", "fdk"):
        vb = host(tg.backproject(g, dev(ys), method))
        for i in range(3):
            np.testing.assert_array_equal(vb[i], host(tg.backproject(g, dev(ys[i]), method)))


def test_host_buffers_equal_device_buffers():
    g = ragged_geometry(14)
    x = inputs.random_volume(g, seed=15)
    y = inputs.random_projections(g, seed=16)
    np.testing.assert_array_equal(tg.forward(g, x, "interp"), host(tg.forward(g, dev(x), "interp")))
    np.testing.assert_array_equal(tg.backproject(g, y, "matched"), host(tg.backproject(g, dev(y), "matched")))
    np.testing.assert_array_equal(tg.fdk(g, y), host(tg.fdk(g, dev(y))))
    # pinned host memory takes the same path
    xp = torch.from_numpy(x).pin_memory()
    np.testing.assert_array_equal(tg.forward(g, xp, "siddon").numpy(), host(tg.forward(g, dev(x), "siddon")))


def test_empty_and_degenerate_inputs():
    g = inputs.circular_geometry((6, 5, 4), (1.0,) * 3, (7, 5), (1.0, 1.0), 3, 100.0, 150.0)
    # no angles: forward is a no-op, backprojection gives zeros
    g0 = g.subset([])
    vol = dev(np.full(g.vol_shape, 7.0))
    out = tg.backproject(g0, torch.zeros((0, 5, 7), device="cuda"), "matched", out=vol)
    assert float(out.abs().max()) == 0.0
    # detector that misses the volume
    gm = inputs.circular_geometry((6, 5, 4), (1.0,) * 3, (7, 5), (1.0, 1.0), 3, 100.0, 150.0)
    gm.offDetector = np.tile([300.0, 0.0], (3, 1))
    for method in ("interp", "siddon"):
        assert float(tg.forward(gm, dev(np.ones(gm.vol_shape)), method).abs().max()) == 0.0
    # one voxel, one pixel
    g1 = inputs.circular_geometry((1, 1, 1), (2.0,) * 3, (1, 1), (1.0, 1.0), 2, 50.0, 80.0)
    x1 = np.full((1, 1, 1), 3.0, np.float32)
    for method in ("interp", "siddon"):
        np.testing.assert_allclose(host(tg.forward(g1, dev(x1), method)), oracle.forward(g1, x1, method),
                                   rtol=1e-6)
    y1 = np.full((2, 1, 1), 2.0, np.float32)
    np.testing.assert_allclose(host(tg.backproject(g1, dev(y1), "matched")), oracle.backproject(g1, y1, "matched"),
                               rtol=1e-6)


def test_rays_on_grid_planes():
    """Rays lying exactly on voxel faces (even sizes, central pixels, angle 0
    and pi/2): the half-open cell rule gives the segment to the upper cell."""
    g = inputs.circular_geometry((8, 8, 8), (1.0,) * 3, (9, 9), (1.0, 1.0), 2, 100.0, 150.0, arc=np.pi)
    x = inputs.random_volume(g, seed=30)
    for method in ("interp", "siddon"):
        assert_proj_close(host(tg.forward(g, dev(x), method)), oracle.forward(g, x, method))


def test_invalid_call_raises():
    g = ragged_geometry()
    g.DSO = np.full(g.nAngles, -1.0)
    with pytest.raises(tg.TgError):
        tg.forward(g, dev(np.zeros(g.vol_shape)), "interp")


# ---------------------------------------------------------------------------
# Full-size workload (512^3, 720 angles, 768 x 1024 detector), in the launch
# configuration the benchmark times: sampled outputs against the oracle and
# the adjoint identity.
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def clinical():
    g = inputs.config_clinical()
    x = inputs.ellipsoid_phantom(g, 40, seed=1)
    return g, x


def test_clinical_forward_sampled_rays(clinical):
    g, x = clinical
    xd = dev(x)
    rng = np.random.default_rng(0)
    rays = np.stack([rng.integers(0, g.nAngles, 300), rng.integers(0, g.nDetector[1], 300),
                     rng.integers(0, g.nDetector[0], 300)], axis=1)
    for method in ("interp", "siddon"):
        p = tg.forward(g, xd, method)
        got = host(p[rays[:, 0], rays[:, 1], rays[:, 2]])
        ref = oracle.forward_rays(g, x, rays, method)
        assert rel_l2(got, ref) <= RTOL_L2, (method, rel_l2(got, ref))
        assert max_rel(got, ref) <= RTOL_MAX
        del p
        torch.cuda.empty_cache()


def test_clinical_backprojections_sampled_voxels(clinical):
    g, _ = clinical
    y = inputs.random_projections(g, seed=3)
    yd = dev(y)
    rng = np.random.default_rng(1)
    vox = np.concatenate([
        np.stack([rng.integers(0, 512, 40), rng.integers(0, 512, 40), rng.integers(0, 512, 40)], axis=1),
        np.array([[0, 0, 0], [511, 511, 511], [0, 255, 300], [256, 0, 10], [100, 200, 511]]),
    ])
    for method in ("matched", "fdk"):
        v = tg.backproject(g, yd, method)
        got = host(v[vox[:, 2], vox[:, 1], vox[:, 0]])
        ref = oracle.backproject_voxels(g, y, vox, method)
        assert rel_l2(got, ref) <= RTOL_L2, (method, rel_l2(got, ref))
        assert max_rel(got, ref) <= RTOL_MAX
        del v
        torch.cuda.empty_cache()


def test_clinical_adjoint_identity(clinical):
    g, x = clinical
    xd = dev(x)
    yd = dev(inputs.random_projections(g, seed=4))
    lhs = float(torch.sum(tg.forward(g, xd, "interp").double() * yd.double()))
    rhs = float(torch.sum(xd.double() * tg.backproject(g, yd, "matched").double()))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_batched_operators_match_per_volume():
    """tg_forward_batched / tg_backproject_batched / tg_gradient_batched on
    volumes of different sizes, detectors, angle counts and geometries give,
    bit for bit, the per-volume results (one launch per operator instead of
    one per volume), and the per-volume results match the oracle."""
    import torch
    geos = [inputs.random_geometry((20, 18, 14), (1.0, 1.1, 0.9), (24, 20), (1.3, 1.2), 8, seed=41),
            inputs.random_geometry((33, 17, 25), (0.8, 1.0, 1.2), (30, 26), (1.1, 1.4), 11, seed=42),
            inputs.circular_geometry((16, 16, 16), (1.5,) * 3, (20, 20), (2.0, 2.0), 5, 400.0, 700.0)]
    rng = np.random.default_rng(43)
    vols = [rng.random(g.vol_shape).astype(np.float32) for g in geos]
    projs = [rng.random(g.proj_shape).astype(np.float32) for g in geos]
    vpk = torch.from_numpy(np.concatenate([v.ravel() for v in vols])).cuda()
    ppk = torch.from_numpy(np.concatenate([p.ravel() for p in projs])).cuda()
    fb = tg.forward_batched(geos, vpk)
    bb = tg.backproject_batched(geos, ppk)
    gb = tg.gradient_batched(geos, vpk, ppk)
    g0 = tg.gradient_batched(geos, vpk, None)
    acc = torch.ones_like(vpk)
    tg.gradient_batched(geos, vpk, ppk, out=acc, accumulate=True)
    po = vo = 0
    for g, v, p in zip(geos, vols, projs):
        nv, np_ = v.size, p.size
        vt, pt = torch.from_numpy(v).cuda(), torch.from_numpy(p).cuda()
        assert torch.equal(fb[po:po + np_].view(g.proj_shape), tg.forward(g, vt, "interp"))
        assert torch.equal(bb[vo:vo + nv].view(g.vol_shape), tg.backproject(g, pt, "matched"))
        gr = tg.gradient(g, vt, pt)
        assert torch.equal(gb[vo:vo + nv].view(g.vol_shape), gr)
        assert torch.equal(g0[vo:vo + nv].view(g.vol_shape), tg.gradient(g, vt, None))
        assert torch.equal(acc[vo:vo + nv].view(g.vol_shape), gr + 1.0)
        assert rel_l2(fb[po:po + np_].cpu().numpy(), oracle.forward(g, v).ravel()) <= 1e-5
        assert rel_l2(bb[vo:vo + nv].cpu().numpy(), oracle.backproject(g, p).ravel()) <= 1e-5
        po += np_
        vo += nv


def test_batched_operators_split_into_chunks():
    """More volumes than one launch's table holds (16) and more slices than
    one texture array holds (2048): the calls split into chunks and still
    agree bit for bit with the per-volume operators."""
    import torch
    geos = [inputs.circular_geometry((6 + k % 3, 5 + k % 2, 4 + k % 4), (1.0,) * 3, (10, 8), (1.5, 1.5), 3 + k % 2,
                                     300.0, 500.0) for k in range(18)]
    geos += [inputs.circular_geometry((3, 3, 1100), (1.0,) * 3, (6, 40), (1.5, 1.5), 2, 2000.0, 3000.0),
             inputs.circular_geometry((3, 2, 1000), (1.0,) * 3, (6, 40), (1.5, 1.5), 2, 2000.0, 3000.0)]
    rng = np.random.default_rng(51)
    vols = [rng.random(g.vol_shape).astype(np.float32) for g in geos]
    projs = [rng.random(g.proj_shape).astype(np.float32) for g in geos]
    vpk = torch.from_numpy(np.concatenate([v.ravel() for v in vols])).cuda()
    ppk = torch.from_numpy(np.concatenate([p.ravel() for p in projs])).cuda()
    fb = tg.forward_batched(geos, vpk)
    bb = tg.backproject_batched(geos, ppk)
    po = vo = 0
    for g, v, p in zip(geos, vols, projs):
        vt, pt = torch.from_numpy(v).cuda(), torch.from_numpy(p).cuda()
        assert torch.equal(fb[po:po + p.size].view(g.proj_shape), tg.forward(g, vt, "interp"))
        assert torch.equal(bb[vo:vo + v.size].view(g.vol_shape), tg.backproject(g, pt, "matched"))
        po += p.size
        vo += v.size


def test_matched_backprojection_propagates_non_finite_data():
    """One Inf and one NaN pixel: the FP64 oracle makes the voxels those rays
    touch non-finite; the fixed-point GPU transpose, which has no scale for
    such data, returns NaN in every voxel (a superset), and CGLS on the same
    data returns NaN instead of finite-looking values."""
    g = ragged_geometry(13)
    y = inputs.random_projections(g, seed=14)
    y[2, 10, 20] = np.inf
    y[5, 7, 3] = np.nan
    ref = oracle.backproject(g, y, "matched")
    bad_ref = ~np.isfinite(ref)
    assert bad_ref.any() and not bad_ref.all()
    got = host(tg.backproject(g, dev(y), "matched"))
    assert np.isnan(got).all()
    yb = dev(np.stack([inputs.random_projections(g, seed=15), y]))
    both = host(tg.backproject(g, yb, "matched"))
    assert np.isnan(both[1]).all()
    assert_vol_close(both[0], oracle.backproject(g, inputs.random_projections(g, seed=15), "matched"))
    assert np.isnan(host(tg.cgls(g, dev(y), 2))).all()


def test_matched_backprojection_wide_dynamic_range():
    """The fixed-point transpose scales every product by one factor from
    max |y|; rays far below the maximum go to a second class 64 times finer.
    With 0.2 % of the rays 1e4 times larger than the rest, the voxels seen
    mostly by the small rays still match the oracle closely."""
    g = ragged_geometry(17)
    rng = np.random.default_rng(33)
    y = (rng.random(g.proj_shape) * 1e-3 + 1e-4).astype(np.float32)
    big = rng.random(g.proj_shape) < 0.002
    y[big] *= 1e4
    got = host(tg.backproject(g, dev(y), "matched"))
    ref = oracle.backproject(g, y, "matched")
    assert_vol_close(got, ref)
    small = np.abs(ref) < np.percentile(np.abs(ref), 20)
    assert rel_l2(got[small], ref[small]) <= 1e-4, rel_l2(got[small], ref[small])
