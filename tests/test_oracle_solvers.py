"""Pins of the oracle's iterative solvers (SIRT / OS-SART, Sec. 2.1 and
Sec. 2.2.2 Eq. 6; CGLS, Sec. 2.1 Krylov methods) on a tiny problem whose
system matrix is materialised column by column, so that the solvers can be
compared with dense linear algebra."""
import numpy as np
import pytest

import oracle
from paper_2412_10129_gb300 import inputs


def tiny_geo(n_angles=3):
    return inputs.circular_geometry((4, 4, 4), (1.0,) * 3, (8, 8), (0.9, 0.9), n_angles, 30.0, 50.0)


def dense_A(g):
    nvox = int(np.prod(g.vol_shape))
    cols = []
    for j in range(nvox):
        e = np.zeros(nvox)
        e[j] = 1.0
        cols.append(oracle.forward(g, e.reshape(g.vol_shape), "interp").reshape(-1))
    return np.stack(cols, axis=1)


@pytest.fixture(scope="module")
def problem():
    g = tiny_geo()
    A = dense_A(g)
    rng = np.random.default_rng(0)
    xt = rng.random(A.shape[1])
    b = A @ xt + 0.01 * rng.standard_normal(A.shape[0])
    return g, A, xt, b


def test_dense_matrix_matches_backprojection(problem):
    g, A, _, _ = problem
    y = np.random.default_rng(1).random(A.shape[0])
    np.testing.assert_allclose(oracle.backproject(g, y.reshape(g.proj_shape), "matched").reshape(-1),
                               A.T @ y, rtol=1e-12, atol=1e-13)


def test_cgls_reaches_least_squares_solution(problem):
    g, A, _, b = problem
    x, hist = oracle.cgls(g, b.reshape(g.proj_shape), 300)
    ref = np.linalg.pinv(A) @ b   # minimum-norm least-squares solution
    assert np.linalg.norm(x.reshape(-1) - ref) / np.linalg.norm(ref) < 1e-6
    assert hist[-1] == pytest.approx(np.linalg.norm(A @ ref - b), rel=1e-8)


def test_cgls_residual_is_monotone(problem):
    g, _, _, b = problem
    _, hist = oracle.cgls(g, b.reshape(g.proj_shape), 40)
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])


def test_cgls_exact_data_and_warm_start(problem):
    """Started at the exact solution of consistent data, CGLS does not move."""
    g, A, xt, _ = problem
    b = A @ xt
    x, hist = oracle.cgls(g, b.reshape(g.proj_shape), 5, x0=xt.reshape(g.vol_shape))
    np.testing.assert_allclose(x.reshape(-1), xt, rtol=0, atol=1e-12)
    assert hist.max() < 1e-10


def dense_sirt(A, b, niter, lam=1.0, nonneg=True, x0=None, floor=0.0):
    """SIRT on a materialised A; a column whose sum is below `floor` (the
    coverage reading: less than 1e-3 of one full-weight sample) gets V = 0."""
    rs, cs = A.sum(1), A.sum(0)
    W = np.where(rs != 0, 1.0 / np.where(rs != 0, rs, 1), 0.0)
    seen = (cs != 0) & (cs >= floor)
    V = np.where(seen, 1.0 / np.where(seen, cs, 1), 0.0)
    x = np.zeros(A.shape[1]) if x0 is None else x0.copy()
    for _ in range(niter):
        x = x + lam * V * (A.T @ (W * (b - A @ x)))
        if nonneg:
            x = np.maximum(x, 0)
    return x


def test_coverage_floor_drops_thin_columns(problem, monkeypatch):
    """V = 0 for a voxel whose column sum is below the coverage floor
    (1e-3 of one sample step by default); raised to the 30th percentile of
    the column sums, the floor removes the thinner columns, and SIRT still
    equals the dense iteration written with the same rule."""
    g, A, _, b = problem
    delta = 0.5 * min(g.dVoxel)
    assert oracle.coverage_floor(g) == pytest.approx(1e-3 * delta, rel=1e-15)
    cs = A.sum(0)
    frac = np.percentile(cs[cs > 0], 30) / delta
    monkeypatch.setattr(oracle, "COVERAGE_MIN", frac)
    floor = frac * delta
    thin = (cs > 0) & (cs < floor)
    assert thin.sum() > 0
    _, V = oracle.sirt_weights(g)
    assert np.all(V.reshape(-1)[thin] == 0.0)
    np.testing.assert_allclose(V.reshape(-1)[cs >= floor], 1.0 / cs[cs >= floor], rtol=1e-10)
    x, _ = oracle.sirt(g, b.reshape(g.proj_shape), 3)
    np.testing.assert_allclose(x.reshape(-1), dense_sirt(A, b, 3, floor=floor), rtol=1e-10, atol=1e-12)


def test_sirt_matches_dense_iteration(problem):
    g, A, _, b = problem
    x, _ = oracle.sirt(g, b.reshape(g.proj_shape), 7, lam=0.9)
    np.testing.assert_allclose(x.reshape(-1), dense_sirt(A, b, 7, lam=0.9), rtol=1e-10, atol=1e-12)


def test_sirt_consistent_data_residual_decreases(problem):
    g, A, xt, _ = problem
    b = A @ xt
    _, hist = oracle.sirt(g, b.reshape(g.proj_shape), 15, nonneg=False)
    assert np.all(np.diff(hist) < 0)


def test_sirt_single_voxel_single_ray():
    """One voxel and one ray: W = V = 1/a so one step gives x = b / a."""
    g = inputs.circular_geometry((1, 1, 1), (2.0,) * 3, (1, 1), (1.0, 1.0), 1, 50.0, 80.0)
    a = float(oracle.forward(g, np.ones((1, 1, 1)), "interp")[0, 0, 0])
    assert a > 0
    x, _ = oracle.sirt(g, np.full((1, 1, 1), 3.0), 1)
    assert x[0, 0, 0] == pytest.approx(3.0 / a, rel=1e-14)


def test_ossart_one_block_is_sirt(problem):
    g, _, _, b = problem
    xs, _ = oracle.sirt(g, b.reshape(g.proj_shape), 3)
    xo, _ = oracle.ossart(g, b.reshape(g.proj_shape), 3, blocksize=g.nAngles)
    np.testing.assert_allclose(xo, xs, rtol=1e-13, atol=1e-15)


def test_ossart_blocks_match_dense(problem):
    g, A, _, b = problem
    nrow = g.nDetector[0] * g.nDetector[1]
    x = np.zeros(A.shape[1])
    for _ in range(2):
        for blk in oracle.subsets(g.nAngles, 2):
            rows = np.concatenate([np.arange(a * nrow, (a + 1) * nrow) for a in blk])
            x = dense_sirt(A[rows], b[rows], 1, x0=x)
    xo, _ = oracle.ossart(g, b.reshape(g.proj_shape), 2, blocksize=2)
    np.testing.assert_allclose(xo.reshape(-1), x, rtol=1e-10, atol=1e-12)


def test_subsets_ragged_tail():
    blocks = oracle.subsets(7, 3)
    assert [list(b) for b in blocks] == [[0, 1, 2], [3, 4, 5], [6]]


def test_oracle_gradient_is_exact_central_difference():
    """The loss ||A x - b||^2 is quadratic, so a central difference equals the
    gradient 2 A^T (A x - b) up to rounding (pins the gradient used to judge
    the differentiable projector)."""
    g = inputs.circular_geometry((8, 7, 6), (1.0,) * 3, (12, 10), (1.0, 1.0), 5, 60.0, 100.0)
    rng = np.random.default_rng(4)
    x, b = rng.random(g.vol_shape), rng.random(g.proj_shape)
    grad = 2 * oracle.backproject(g, oracle.forward(g, x, "interp") - b, "matched")
    h = 1e-3
    for j in rng.choice(x.size, 12, replace=False):
        e = np.zeros(x.size)
        e[j] = h
        e = e.reshape(x.shape)
        fp = np.sum((oracle.forward(g, x + e, "interp") - b) ** 2)
        fm = np.sum((oracle.forward(g, x - e, "interp") - b) ** 2)
        assert (fp - fm) / (2 * h) == pytest.approx(grad.reshape(-1)[j], rel=1e-6, abs=1e-9)
