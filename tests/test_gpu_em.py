"""GPU parity of the Siddon transpose and of MLEM / OS-EM (Sec. 2.1, Eq. 5)
against the FP64 oracle, through the C ABI.

Tolerances: the Siddon transpose as the other backprojectors (relative L2
<= 1e-5, max-abs <= 1e-4 of the maximum); MLEM / OS-EM after their
iterations <= 1e-4 relative L2, the bar of the iterative solvers (FP32
iterates, each update a product of FP32 projector outputs)."""
import numpy as np
import pytest

import oracle
from conftest import max_rel, rel_l2
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


def ragged_geometry(seed=3):
    return inputs.random_geometry((37, 29, 23), (1.0, 1.2, 0.9), (45, 31), (1.3, 1.1), 13, seed=seed,
                                  DSO=300.0, DSD=520.0)


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_siddon_transpose_matches_oracle(which):
    g = inputs.config_small() if which == "small" else ragged_geometry()
    y = inputs.random_projections(g, seed=31)
    got = host(tg.backproject(g, dev(y), "siddon"))
    ref = oracle.backproject(g, y, "siddon")
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)
    assert max_rel(got, ref) <= 1e-4, max_rel(got, ref)


def test_siddon_adjoint_identity():
    """<A x, y> = <x, A^T y> for the GPU pair, FP64 inner products."""
    g = ragged_geometry(5)
    x = inputs.random_volume(g, seed=32)
    y = inputs.random_projections(g, seed=33)
    Ax = host(tg.forward(g, dev(x), "siddon"))
    Aty = host(tg.backproject(g, dev(y), "siddon"))
    lhs = float(np.sum(Ax * y.astype(np.float64)))
    rhs = float(np.sum(x.astype(np.float64) * Aty))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_siddon_transpose_batch_host_and_noalloc():
    """A batch of two projection sets in one launch, host buffers and the
    allocation-free entry point give the per-call results (FP32 reductions
    in a varying order: equal to rounding, not bit for bit)."""
    g = ragged_geometry(7)
    y = np.stack([inputs.random_projections(g, seed=34), inputs.random_projections(g, seed=35)])
    bat = host(tg.backproject(g, dev(y), "siddon"))
    for k in range(2):
        one = host(tg.backproject(g, dev(y[k]), "siddon"))
        assert rel_l2(bat[k], one) <= 1e-6
        hst = tg.backproject(g, y[k].astype(np.float32), "siddon").astype(np.float64)
        assert rel_l2(hst, one) <= 1e-6
        na = host(tg.backproject_noalloc(g, dev(y[k]), "siddon"))
        assert rel_l2(na, one) <= 1e-6


@pytest.fixture(scope="module")
def em_problem():
    g = inputs.config_small()
    x = inputs.ellipsoid_phantom(g, 10, seed=1)
    b = oracle.forward(g, x, "interp")
    bs = oracle.forward(g, x, "siddon")
    return g, b, bs


@pytest.mark.parametrize("method", ["interp", "siddon"])
def test_mlem_matches_oracle(em_problem, method):
    g, b, bs = em_problem
    data = b if method == "interp" else bs
    n = 20
    x, h = tg.mlem(g, dev(data), n, method=method, resid=True)
    xr, hr = oracle.mlem(g, data, n, method=method)
    assert rel_l2(host(x), xr) <= 1e-4, rel_l2(host(x), xr)
    np.testing.assert_allclose(h, hr, rtol=1e-4)
    assert hr[-1] < 0.5 * hr[0]


@pytest.mark.parametrize("method", ["interp", "siddon"])
def test_osem_matches_oracle(em_problem, method):
    g, b, bs = em_problem
    data = b if method == "interp" else bs
    x, h = tg.osem(g, dev(data), 5, blocksize=20, method=method, resid=True)
    xr, hr = oracle.osem(g, data, 5, 20, method=method)
    assert rel_l2(host(x), xr) <= 1e-4, rel_l2(host(x), xr)
    np.testing.assert_allclose(h, hr, rtol=1e-4)


def test_osem_ragged_blocks_and_warm_start():
    """Blocks of 4 over 13 angles (the last holds one), a given positive x0,
    arbitrary per-angle geometry."""
    g = ragged_geometry(9)
    x0 = np.random.default_rng(36).uniform(0.5, 1.5, g.vol_shape)
    b = oracle.forward(g, inputs.random_volume(g, seed=37))
    x = tg.osem(g, dev(b), 3, blocksize=4, x0=dev(x0))
    xr, _ = oracle.osem(g, b, 3, 4, x0=x0.astype(np.float32))
    assert rel_l2(host(x), xr) <= 1e-4, rel_l2(host(x), xr)


def test_mlem_conserves_counts_on_gpu():
    """One GPU MLEM update: sum_j (A^T 1)_j x_j = sum of b over rays with A x0 != 0."""
    g = inputs.config_small()
    b = inputs.random_projections(g, seed=38).astype(np.float64) + 0.5
    x1 = host(tg.mlem(g, dev(b), 1))
    s = oracle.backproject(g, np.ones(g.proj_shape), "matched")
    seen = oracle.forward(g, np.ones(g.vol_shape)) != 0
    assert np.sum(s * x1) == pytest.approx(np.sum(b[seen]), rel=1e-5)


def test_osem_random_order_matches_oracle(em_problem):
    g, b, _ = em_problem
    x = tg.osem(g, dev(b), 2, blocksize=20, order="random", seed=11)
    xr, _ = oracle.osem(g, b, 2, 20, order="random", seed=11)
    assert rel_l2(host(x), xr) <= 1e-4, rel_l2(host(x), xr)
