"""Chirp-time rectangle tiling (Sec. IV): the host helper fcas_tau_tiles, checked against the
definition of an overlapping cover (no GPU needed: the function is host code in libfcas.so)."""

import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def fc():
    from paper_2002_02150_gb300 import build as b
    b.build()
    import paper_2002_02150_gb300 as mod
    return mod


@pytest.mark.parametrize("n0,n15,ov", [(1, 1, 0.0), (3, 2, 0.0), (4, 5, 0.25), (7, 1, 0.5), (2, 9, 0.9)])
def test_tiles_cover_the_rectangle_with_the_stated_overlap(fc, n0, n15, ov):
    lo0, hi0, lo15, hi15 = 2.5, 14.75, 0.265, 0.552
    b = fc.fcas_tau_tiles(lo0, hi0, lo15, hi15, n0, n15, ov).reshape(n0, n15, 8)
    # whole sky in every tile
    assert np.all(b[..., 0] == 0.0) and np.allclose(b[..., 1], 2 * math.pi)
    assert np.allclose(b[..., 2], -0.5 * math.pi) and np.allclose(b[..., 3], 0.5 * math.pi)
    for axis, (lo, hi, n, k) in enumerate(((lo0, hi0, n0, 4), (lo15, hi15, n15, 6))):
        tiles = b[:, 0, k:k + 2] if axis == 0 else b[0, :, k:k + 2]
        w = (hi - lo) / (n - (n - 1) * ov)
        assert tiles[0, 0] == lo and tiles[-1, 1] == hi
        np.testing.assert_allclose(tiles[:, 1] - tiles[:, 0], w, rtol=1e-12)
        # neighbours share exactly the fraction `ov` of a width; no gaps
        np.testing.assert_allclose(tiles[:-1, 1] - tiles[1:, 0], ov * w, rtol=1e-9, atol=1e-12)
        # every point of the range lies in some tile
        pts = np.linspace(lo, hi, 1001)
        inside = (pts[:, None] >= tiles[None, :, 0] - 1e-12) & (pts[:, None] <= tiles[None, :, 1] + 1e-12)
        assert inside.any(axis=1).all()
    # rows vary tau1.5 fastest: tile (j0, j15) at index j0 * n15 + j15
    assert np.all(b[:, :, 4] == b[:, :1, 4]) and np.all(b[:, :, 6] == b[:1, :, 6])


@pytest.mark.parametrize("args", [(2.0, 1.0, 0.1, 0.2, 2, 2, 0.0), (1.0, 2.0, 0.1, 0.2, 0, 2, 0.0),
                                  (1.0, 2.0, 0.1, 0.2, 2, 2, 1.0), (0.0, 2.0, 0.1, 0.2, 2, 2, 0.0),
                                  (1.0, float("nan"), 0.1, 0.2, 2, 2, 0.0)])
def test_invalid_tilings_are_rejected(fc, args):
    with pytest.raises(fc.FcasError):
        fc.fcas_tau_tiles(*args)
