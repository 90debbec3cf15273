"""The seeded synthetic workloads (phantoms.py): shapes, value ranges, the
hyperparameters each workload is run with, and reproducibility from the seed.
These are the inputs every parity test and the benchmark use."""
import numpy as np
import pytest

import phantoms


def _check(w, ndim, dims, B, T, sigma):
    assert w.ndim == ndim and tuple(w.dims) == tuple(dims) and w.T == T and w.sigma == sigma
    for a in (w.I0, w.J, w.p0):
        assert a.shape == (B,) + tuple(dims) and a.dtype == np.float32
        assert a.flags["C_CONTIGUOUS"] and np.isfinite(a).all()
    for a in (w.mu, w.rho, w.lam):
        assert a.shape == (B,) and a.dtype == np.float32
    # images are clipped to [0, 1]
    assert w.I0.min() >= 0.0 and w.I0.max() <= 1.0
    assert w.J.min() >= 0.0 and w.J.max() <= 1.0
    assert np.all(w.rho == 1.0)


def test_disk_pair():
    """64^2 disk of radius 18 -> ellipse plus a blob at (52, 32), outside the ellipse
    and the disk; T = 10, sigma = 3, mu = 0.1, lambda = 1e-3; p0 ~ N(0, 0.01^2) or 0."""
    w = phantoms.disk_pair_64()
    _check(w, 2, (64, 64), 1, 10, 3.0)
    assert w.mu[0] == np.float32(0.1) and w.lam[0] == np.float32(1e-3)
    I, J = w.I0[0], w.J[0]
    assert I[32, 32] > 0.99 and I[32, 32 + 17] > 0.5 and I[32, 32 + 20] < 0.05
    assert J[52, 32] > 0.99 and I[52, 32] < 0.05   # the blob the source lacks
    assert J[32, 32 + 20] > 0.5 and J[32 - 20, 32] < 0.05  # semi-axes 14 (axis 0) x 22
    assert 0.008 < w.p0.std() < 0.012
    assert np.all(phantoms.disk_pair_64(random_p0=False).p0 == 0.0)


def test_c_pair_is_a_disk_and_an_open_ring():
    w = phantoms.c_pair_64()
    _check(w, 2, (64, 64), 1, 20, 3.0)
    assert w.mu[0] == 0.0 and np.all(w.p0 == 0.0)
    c = 31.5
    J = w.J[0]
    assert J[int(c), int(c)] < 0.05                       # the hole of the ring
    assert J[int(c), int(c - 0.27 * 64)] > 0.9            # the ring on the closed side
    assert J[int(c), int(c + 0.27 * 64)] < 0.05           # the gap on the axis-1 side


def test_ellipse_batch():
    """16 pairs of 256^2, T = 20, sigma = 6, mu cycling through 0, 0.05, 0.2."""
    w = phantoms.ellipse_pairs()
    _check(w, 2, (256, 256), 16, 20, 6.0)
    np.testing.assert_array_equal(w.mu, np.float32([0.0, 0.05, 0.2] * 5 + [0.0]))
    assert np.all(w.lam == np.float32(1e-3)) and np.all(w.p0 == 0.0)
    for b in range(16):
        assert w.I0[b].max() > 0.2 and (w.I0[b] > 0.1).mean() > 0.02
        assert not np.array_equal(w.I0[b], w.J[b])
    assert len({w.I0[b].tobytes() for b in range(16)}) == 16


@pytest.mark.parametrize("make", [phantoms.disk_pair_64, phantoms.ellipse_pairs,
                                  lambda seed: phantoms.head_pair_3d(dims=(32, 36, 40),
                                                                     seed=seed)])
def test_workloads_follow_their_seed(make):
    a, b = make(seed=7), make(seed=7)
    c = make(seed=8)
    for x, y in ((a.I0, b.I0), (a.J, b.J), (a.p0, b.p0)):
        np.testing.assert_array_equal(x, y)
    # the disk pair draws only p0; the others draw their images too
    assert not (np.array_equal(a.J, c.J) and np.array_equal(a.p0, c.p0))


def test_head_volume():
    """128^3 nested ellipsoids (0.5 / 0.9 / 0.1), the target warped by at most 4 voxels
    plus a blob; T = 20, sigma = 5, mu = 0.1."""
    w = phantoms.head_pair_3d()
    _check(w, 3, (128, 128, 128), 1, 20, 5.0)
    assert w.mu[0] == np.float32(0.1)
    levels = set(np.round(np.unique(w.I0[0]).astype(np.float64), 2).tolist())
    assert {0.0, 0.1, 0.5, 0.9} <= levels and w.I0.max() <= np.float32(0.9)
    assert np.abs(w.J[0] - w.I0[0]).max() > 0.3


def test_mri_volume_and_its_block_average():
    """160x192x160 with Rician-like noise (strictly positive), T = 20, sigma = 6,
    mu = 0.05, lambda = 1e-4; its 2x block average keeps the mean."""
    w = phantoms.mri_pair_3d()
    _check(w, 3, (160, 192, 160), 1, 20, 6.0)
    assert w.mu[0] == np.float32(0.05) and w.lam[0] == np.float32(1e-4)
    assert w.I0.min() > 0.0 and w.J.min() > 0.0
    small = phantoms.block_average(w.I0)
    assert small.shape == (1, 80, 96, 80) and small.dtype == np.float32
    assert abs(float(small.mean()) - float(w.I0.mean())) < 1e-6
    np.testing.assert_allclose(small[0, 3, 4, 5], w.I0[0, 6:8, 8:10, 10:12].mean(), rtol=1e-6)


def test_mixed_batch():
    """64 pairs with sizes from {96^2, 160^2, 224^2, 64^3, 96^3}, T in {10, 15, 20},
    sigma in [2, 6], mu in [0, 0.2]; both dimensions present."""
    ws = phantoms.mixed_pairs()
    assert len(ws) == 64
    sizes = {tuple(w.dims) for w in ws}
    assert sizes <= {(96, 96), (160, 160), (224, 224), (64, 64, 64), (96, 96, 96)}
    assert {len(d) for d in sizes} == {2, 3}
    for w in ws:
        assert w.I0.shape[0] == 1 and w.T in (10, 15, 20) and 2.0 <= w.sigma <= 6.0
        assert 0.0 <= w.mu[0] <= 0.2 and w.I0.min() >= 0.0 and w.I0.max() <= 1.0
