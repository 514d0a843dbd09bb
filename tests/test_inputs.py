"""The synthetic inputs: SU(3) links, APE smoothing, sources."""
import numpy as np

from paper_1011_2775_gb300 import inputs as I


def _plaquette(U):
    dag = lambda m: np.conj(np.swapaxes(m, -1, -2))  # noqa: E731
    tot, n = 0.0, 0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            um, un = U[..., mu, :, :], U[..., nu, :, :]
            p = um @ np.roll(un, -1, axis=3 - mu) @ dag(np.roll(um, -1, axis=3 - nu)) @ dag(un)
            tot += np.trace(p, axis1=-2, axis2=-1).real.mean() / 3
            n += 1
    return tot / n


def test_links_are_su3_and_ape_smooths():
    dims = (4, 4, 4, 4)
    U0 = I.make_gauge(dims, 0.25, 0, 0.5, 2001)
    U5 = I.make_gauge(dims, 0.25, 5, 0.5, 2001)
    for U in (U0, U5):
        uu = np.conj(np.swapaxes(U, -1, -2)) @ U
        assert np.abs(uu - np.eye(3)).max() < 1e-13
        assert np.abs(np.linalg.det(U) - 1).max() < 1e-13
    assert _plaquette(U5) > _plaquette(U0) > 0.5
    # seeded: same seed, same field
    assert np.array_equal(U0, I.make_gauge(dims, 0.25, 0, 0.5, 2001))


def test_sources():
    dims = (4, 4, 4, 8)
    g = I.gaussian_source(dims, 3)
    assert g.shape == (8, 4, 4, 4, 4, 3)
    assert abs(g.real.var() - 0.5) < 0.05
    p = I.point_source(dims, 7, site=(1, 2, 3, 4))
    assert p[4, 3, 2, 1, 2, 1] == 1 and np.count_nonzero(p) == 1
    G = I.random_gauge_transform(dims, 5)
    assert np.abs(np.conj(np.swapaxes(G, -1, -2)) @ G - np.eye(3)).max() < 1e-13
