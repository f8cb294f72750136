"""Pins of the oracle's LSMR (Sec. 2.1, Krylov methods; Fong and Saunders):
its k-th iterate minimises ||A^T (b - A x)|| over the Krylov space
K_k(A^T A, A^T b), checked against an explicit Krylov basis and numpy's
least squares on a materialised small A; ||A^T r_k|| decreases; n
iterations reach the least-squares solution."""
import numpy as np
import pytest

import oracle
from paper_2412_10129_gb300 import inputs


def _geo():
    # 8 views: A has full column rank (condition number ~29)
    return inputs.random_geometry((5, 4, 3), (1.0, 1.1, 0.9), (7, 5), (1.2, 1.0), 8, seed=71, DSO=150.0, DSD=250.0)


@pytest.fixture(scope="module")
def dense():
    g = _geo()
    n = int(np.prod(g.vol_shape))
    A = np.stack([oracle.forward(g, e.reshape(g.vol_shape)).ravel() for e in np.eye(n)], axis=1)
    At = np.stack([oracle.backproject(g, e.reshape(g.proj_shape), "matched").ravel()
                   for e in np.eye(A.shape[0])], axis=1)
    b = np.random.default_rng(72).uniform(0, 1, g.proj_shape)
    return g, A, At, b


def test_lsmr_iterates_minimise_the_normal_residual_over_the_krylov_space(dense):
    g, A, At, b = dense
    N = At @ A
    c = At @ b.ravel()
    K = [c / np.linalg.norm(c)]
    for k in range(1, 6):
        x, _ = oracle.lsmr(g, b, k)
        V = np.stack(K, axis=1)
        y = np.linalg.lstsq(N @ V, c, rcond=None)[0]
        ref = V @ y
        assert np.linalg.norm(x.ravel() - ref) <= 1e-8 * np.linalg.norm(ref), k
        # extend the orthonormal Krylov basis by one vector
        q = N @ K[-1]
        for w in K:
            q = q - (w @ q) * w
        K.append(q / np.linalg.norm(q))


def test_lsmr_normal_residual_decreases_and_reaches_least_squares(dense):
    g, A, At, b = dense
    n = A.shape[1]
    prev = np.inf
    for k in (1, 2, 4, 8, 16):
        x, _ = oracle.lsmr(g, b, k)
        nr = np.linalg.norm(At @ (b.ravel() - A @ x.ravel()))
        assert nr <= prev * (1 + 1e-12)
        prev = nr
    x, h = oracle.lsmr(g, b, 3 * n)
    ref = np.linalg.lstsq(A, b.ravel(), rcond=None)[0]
    assert np.linalg.norm(x.ravel() - ref) <= 1e-6 * np.linalg.norm(ref)
    assert h[-1] == pytest.approx(np.linalg.norm(b.ravel() - A @ ref), rel=1e-8)
