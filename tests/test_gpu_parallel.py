"""GPU parity of the parallel-beam mode (the synchrotron shapes of Sec. 3)
against the FP64 oracle, through the C ABI: both projectors, both
transposes, parallel FBP, CGLS, the adjoint identity and the batched calls.
Tolerances as for the cone beam (relative L2 <= 1e-5 per projection and
volume, max-abs <= 1e-4 of the maximum; 1e-4 after iterations)."""
import math

import numpy as np
import pytest

import oracle
from conftest import max_rel, rel_l2
from oracle import fdk_variants as ofdk
from paper_2412_10129_gb300 import inputs, tg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def close(got, ref, tol=1e-5):
    assert rel_l2(got, ref) <= tol, rel_l2(got, ref)
    assert max_rel(got, ref) <= 10 * tol, max_rel(got, ref)


def par_geometry(seed=11, n=17, tilt=True):
    """Parallel scan with per-angle detector offsets, tilts and COR."""
    g = inputs.parallel_geometry((37, 29, 23), (1.0, 1.2, 0.9), (45, 31), (1.1, 1.0), n, arc=math.pi,
                                 DSO=300.0, DSD=520.0)
    rng = np.random.default_rng(seed)
    g.offDetector = rng.uniform(-2, 2, size=(n, 2))
    g.COR = rng.uniform(-1, 1, size=n)
    if tilt:
        g.rotDetector = rng.uniform(-0.03, 0.03, size=(n, 3))
    return g


@pytest.mark.parametrize("method", ["interp", "siddon"])
def test_parallel_forward_matches_oracle(method):
    g = par_geometry()
    x = inputs.random_volume(g, seed=12)
    close(host(tg.forward(g, dev(x), method)), oracle.forward(g, x, method))


@pytest.mark.parametrize("bp", ["matched", "siddon"])
def test_parallel_backprojections_match_oracle(bp):
    g = par_geometry(13)
    y = inputs.random_projections(g, seed=14)
    close(host(tg.backproject(g, dev(y), bp)), oracle.backproject(g, y, bp))


@pytest.mark.parametrize("method,bp", [("interp", "matched"), ("siddon", "siddon")])
def test_parallel_adjoint_identity(method, bp):
    g = par_geometry(15)
    x = inputs.random_volume(g, seed=16)
    y = inputs.random_projections(g, seed=17)
    lhs = float(np.sum(host(tg.forward(g, dev(x), method)) * y.astype(np.float64)))
    rhs = float(np.sum(x.astype(np.float64) * host(tg.backproject(g, dev(y), bp))))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_parallel_fbp_matches_oracle():
    g = inputs.parallel_geometry((48, 48, 16), (1.0,) * 3, (96, 20), (0.75, 1.0), 90, arc=math.pi)
    b = oracle.forward(g, inputs.ellipsoid_phantom(g, 6, seed=18), "siddon")
    close(host(tg.fdk(g, dev(b))), oracle.fdk(g, b))
    close(host(tg.fdk_filter(g, dev(b), "hamming")), ofdk.fdk_filter(g, b, "hamming"))


def test_parallel_cgls_matches_oracle():
    g = par_geometry(19, n=24, tilt=False)
    b = oracle.forward(g, inputs.ellipsoid_phantom(g, 5, seed=20, semi_axes=(2.0, 8.0)), "siddon")
    x, h = tg.cgls(g, dev(b), 10, resid=True)
    xr, hr = oracle.cgls(g, b, 10)
    assert rel_l2(host(x), xr) <= 1e-4
    np.testing.assert_allclose(h, hr, rtol=1e-4)


def test_parallel_batched_calls_and_refusals():
    """Batched projector calls over parallel geometries equal the single
    calls; a batch mixing beam modes and Parker / Wang weights on a parallel
    scan are refused."""
    geos = [par_geometry(21 + k, n=5 + k) for k in range(3)]
    vols = [inputs.random_volume(g, seed=30 + k) for k, g in enumerate(geos)]
    vpk = dev(np.concatenate([v.ravel() for v in vols]))
    fb = tg.forward_batched(geos, vpk)
    off = 0
    for g, v in zip(geos, vols):
        n = int(np.prod(g.proj_shape))
        assert torch.equal(fb[off:off + n].view(g.proj_shape), tg.forward(g, dev(v), "interp"))
        off += n
    cone = inputs.circular_geometry(geos[0].nVoxel, geos[0].dVoxel, geos[0].nDetector, geos[0].dDetector, 5,
                                    300.0, 520.0)
    with pytest.raises(tg.TgError):
        tg.forward_batched([geos[0], cone], dev(np.concatenate([vols[0].ravel(), vols[0].ravel()])))
    b = dev(inputs.random_projections(geos[0], seed=40))
    with pytest.raises(tg.TgError):
        tg.fdk(geos[0], b, wang=True)
