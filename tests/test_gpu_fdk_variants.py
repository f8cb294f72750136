"""GPU parity of the FDK variants (Sec. 2.1, direct methods: filter types,
Parker and Wang weights) against the FP64 oracle, through the C ABI.

Tolerances as for the projectors: relative L2 <= 1e-5 per projection and per
volume, max-abs <= 1e-4 of the reference maximum.  The FP32 row filter sums
up to nu - 1 tap pairs (~1e-6 relative) and the FP32 pre-weights carry
~1e-7 relative error each."""
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


def assert_close(got, ref, per_first_axis=True):
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)
    assert max_rel(got, ref) <= 1e-4, max_rel(got, ref)
    if per_first_axis:
        norms = np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)
        for a in np.nonzero(norms > 1e-3 * norms.max())[0]:
            assert rel_l2(got[a], ref[a]) <= 1e-5, (a, rel_l2(got[a], ref[a]))


@pytest.mark.parametrize("name", ofdk.WINDOWS)
@pytest.mark.parametrize("nu", [1, 2, 10, 301, 1024])
def test_filter_windows_match_oracle(name, nu):
    """Every window on rows of 1 to 1024 pixels (ragged against the 9
    outputs a thread makes), arbitrary per-angle geometry with tilted and
    displaced detectors."""
    g = inputs.random_geometry((8, 8, 8), (1.0,) * 3, (nu, 5), (0.9, 1.1), 4, seed=nu)
    p = inputs.random_projections(g, seed=5) - 0.3
    got = host(tg.fdk_filter(g, dev(p), name))
    assert_close(got, ofdk.fdk_filter(g, p, name))


def _short_scan(n_angles=120, arc_deg=200.0):
    g = inputs.config_small()
    arc = math.radians(arc_deg)
    return inputs.circular_geometry(g.nVoxel, g.dVoxel, g.nDetector, g.dDetector, n_angles,
                                    1000.0, 1536.0, arc=arc * n_angles / (n_angles - 1))


def _offset_geometry(n_angles=100, shift_px=40):
    g = inputs.config_small()
    g = inputs.circular_geometry(g.nVoxel, g.dVoxel, g.nDetector, g.dDetector, n_angles, 1000.0, 1536.0)
    g.offDetector[:, 0] = shift_px * g.dDetector[0]
    return g


@pytest.mark.parametrize("name", ["ram-lak", "hamming"])
def test_parker_short_scan_matches_oracle(name):
    """200-degree scan: the Parker-weighted filtered projections and the
    reconstruction (angle weight beta_max / (nAngles - 1))."""
    g = _short_scan()
    x = inputs.ellipsoid_phantom(g, 10, seed=7)
    b = oracle.forward(g, x)
    assert_close(host(tg.fdk_filter(g, dev(b), name, parker=True)), ofdk.fdk_filter(g, b, name, parker=True))
    assert_close(host(tg.fdk(g, dev(b), name, parker=True)), ofdk.fdk(g, b, name, parker=True),
                 per_first_axis=False)


@pytest.mark.parametrize("name", ["ram-lak", "shepp-logan"])
def test_wang_displaced_detector_matches_oracle(name):
    g = _offset_geometry(60, 40)
    x = inputs.ellipsoid_phantom(g, 10, seed=8)
    b = oracle.forward(g, x)
    assert_close(host(tg.fdk_filter(g, dev(b), name, wang=True)), ofdk.fdk_filter(g, b, name, wang=True))
    assert_close(host(tg.fdk(g, dev(b), name, wang=True)), ofdk.fdk(g, b, name, wang=True),
                 per_first_axis=False)


def test_windowed_fdk_matches_oracle():
    """The full-orbit FDK with each window on the 64^3 workload geometry."""
    g = inputs.config_small()
    x = inputs.ellipsoid_phantom(g, 10, seed=1)
    b = oracle.forward(g, x)
    for name in ("shepp-logan", "cosine", "hann"):
        assert_close(host(tg.fdk(g, dev(b), name)), ofdk.fdk(g, b, name), per_first_axis=False)


def test_ramlak_filter_matches_spatial_oracle_on_wide_rows():
    """The ramp on 2048-pixel rows (taps up to 2047) against the C oracle's
    spatial filter, host buffers through the same call."""
    g = inputs.circular_geometry((8, 8, 8), (1.0,) * 3, (2048, 3), (0.2, 0.2), 3, 1000.0, 1536.0)
    p = inputs.random_projections(g, seed=9)
    got = np.zeros(g.proj_shape, np.float32)
    tg.fdk_filter(g, p.astype(np.float32), "ram-lak", out=got)
    assert_close(got.astype(np.float64), oracle.fdk_filter(g, p))
