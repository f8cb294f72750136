"""Pins of the oracle's LSQR (Sec. 2.1, Krylov methods; Paige and Saunders):
LSQR and CGLS build the same Krylov iterates in exact arithmetic, so the
two oracle solvers (written independently) must agree; n iterations on a
materialised small A reach numpy's least-squares solution; the recurrence's
residual estimate phibar is the true ||b - A x_k||."""
import numpy as np
import pytest

import oracle
from paper_2412_10129_gb300 import inputs


def _geo():
    return inputs.random_geometry((5, 4, 3), (1.0, 1.1, 0.9), (7, 5), (1.2, 1.0), 3, seed=61, DSO=150.0, DSD=250.0)


def test_lsqr_iterates_equal_cgls_iterates():
    g = _geo()
    b = np.random.default_rng(62).uniform(0, 1, g.proj_shape)
    for k in (1, 2, 5, 9):
        x1, _ = oracle.lsqr(g, b, k)
        x2, _ = oracle.cgls(g, b, k)
        assert np.linalg.norm(x1 - x2) <= 1e-9 * np.linalg.norm(x2)


def test_lsqr_reaches_the_least_squares_solution():
    g = _geo()
    n = int(np.prod(g.vol_shape))
    A = np.stack([oracle.forward(g, e.reshape(g.vol_shape)).ravel() for e in np.eye(n)], axis=1)
    b = np.random.default_rng(63).uniform(0, 1, g.proj_shape)
    ref = np.linalg.lstsq(A, b.ravel(), rcond=None)[0]
    x, _ = oracle.lsqr(g, b, 3 * n)
    assert np.linalg.norm(x.ravel() - ref) <= 1e-6 * np.linalg.norm(ref)


def test_residual_estimate_is_the_true_residual():
    g = _geo()
    b = np.random.default_rng(64).uniform(0, 1, g.proj_shape)
    x0 = np.random.default_rng(65).uniform(0, 1, g.vol_shape)
    for k in (1, 4, 8):
        x, h = oracle.lsqr(g, b, k, x0=x0)
        assert h[-1] == pytest.approx(np.linalg.norm(b - oracle.forward(g, x)), rel=1e-9)
        assert np.all(np.diff(h) <= 1e-12 * h[0])
