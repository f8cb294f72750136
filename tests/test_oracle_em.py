"""Pins of the oracle's MLEM (Sec. 2.1, Eq. 5) and OS-EM: properties of the
EM update that hold exactly whatever the system matrix -- count (flux)
conservation after every (sub)iteration, consistent data as a fixed point,
the monotone Poisson likelihood (Shepp and Vardi 1982), the one-voxel
closed form -- plus OS-EM with one block = MLEM."""
import numpy as np
import pytest

import oracle
from paper_2412_10129_gb300 import inputs

BP = {"interp": "matched", "siddon": "siddon"}


def _geo(n_angles=6):
    return inputs.random_geometry((11, 9, 7), (1.0, 1.1, 0.9), (15, 12), (1.2, 1.0), n_angles, seed=21,
                                  DSO=200.0, DSD=330.0)


def _data(g, seed=22):
    return np.random.default_rng(seed).uniform(0.5, 2.0, g.proj_shape)


@pytest.mark.parametrize("method", ["interp", "siddon"])
def test_mlem_conserves_counts(method):
    """sum_j (A^T 1)_j x_j after an update = sum of b_i over the rays with
    (A x)_i != 0, for any positive x before it."""
    g = _geo()
    b = _data(g)
    x0 = np.random.default_rng(23).uniform(0.2, 1.0, g.vol_shape)
    x1, _ = oracle.mlem(g, b, 1, x0=x0, method=method)
    s = oracle.backproject(g, np.ones(g.proj_shape), BP[method])
    seen = oracle.forward(g, x0, method) != 0
    assert np.sum(s * x1) == pytest.approx(np.sum(b[seen]), rel=1e-12)


@pytest.mark.parametrize("method", ["interp", "siddon"])
def test_osem_conserves_counts_per_block(method):
    g = _geo(7)
    b = _data(g)
    x = np.random.default_rng(24).uniform(0.2, 1.0, g.vol_shape)
    for idx in oracle.subsets(g.nAngles, 3):
        gs = g.subset(idx)
        seen = oracle.forward(gs, x, method) != 0
        x_next, _ = oracle.osem(gs, b[idx], 1, len(idx), x0=x, method=method)
        s = oracle.backproject(gs, np.ones(gs.proj_shape), BP[method])
        assert np.sum(s * x_next) == pytest.approx(np.sum(b[idx][seen]), rel=1e-12)
        x = x_next


@pytest.mark.parametrize("method", ["interp", "siddon"])
def test_consistent_data_is_a_fixed_point(method):
    g = _geo()
    xs = np.random.default_rng(25).uniform(0.5, 1.5, g.vol_shape)
    b = oracle.forward(g, xs, method)
    x, hist = oracle.osem(g, b, 3, 2, x0=xs, method=method)
    np.testing.assert_allclose(x, xs, rtol=1e-12)
    assert hist[-1] <= 1e-11 * np.linalg.norm(b)


def test_voxels_a_block_does_not_see_keep_their_value():
    """A block of one view sees only part of the volume; the others' values
    pass through its update unchanged."""
    g = _geo(2)
    g1 = g.subset([0])
    unseen = oracle.backproject(g1, np.ones(g1.proj_shape), "matched") == 0
    assert unseen.any()
    x0 = np.random.default_rng(28).uniform(0.2, 1.0, g.vol_shape)
    x, _ = oracle.osem(g1, _data(g1), 1, 1, x0=x0)
    np.testing.assert_array_equal(x[unseen], x0[unseen])


@pytest.mark.parametrize("method", ["interp", "siddon"])
def test_mlem_increases_poisson_likelihood(method):
    """EM never decreases sum_i b_i log(Ax)_i - (Ax)_i (inconsistent data)."""
    g = _geo()
    b = _data(g, 26)
    x = np.ones(g.vol_shape)
    L = [oracle.poisson_loglik(g, x, b, method)]
    for _ in range(12):
        x, _ = oracle.mlem(g, b, 1, x0=x, method=method)
        L.append(oracle.poisson_loglik(g, x, b, method))
    d = np.diff(L)
    assert np.all(d >= -1e-12 * np.abs(L[0])), d
    assert L[-1] > L[0]
    assert np.all(x >= 0)


def test_single_voxel_single_ray():
    """One voxel seen by one ray: x1 = b / a with a the ray's weight."""
    g = inputs.circular_geometry((1, 1, 1), (2.0,) * 3, (1, 1), (0.5, 0.5), 1, 100.0, 150.0)
    for method in ("interp", "siddon"):
        a = oracle.forward(g, np.ones(g.vol_shape), method)[0, 0, 0]
        assert a > 0
        x, _ = oracle.mlem(g, np.full(g.proj_shape, 3.0), 1, method=method)
        assert x[0, 0, 0] == pytest.approx(3.0 / a, rel=1e-13)


def test_osem_with_one_block_is_mlem():
    g = _geo()
    b = _data(g, 27)
    a, ha = oracle.osem(g, b, 4, g.nAngles)
    m, hm = oracle.mlem(g, b, 4)
    np.testing.assert_array_equal(a, m)
    np.testing.assert_array_equal(ha, hm)
