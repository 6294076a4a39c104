"""Pins for the oracle's HEALPix RING pixel centres.

The oracle writes the RING-scheme ring formulas of Gorski et al. (2005).  These
tests check them against facts that do not come from those formulas:

* the 12 base-resolution centres (Nside = 1) are the textbook layout: four at
  z = 2/3 and longitudes pi/4 + k pi/2, four on the equator at k pi/2, four at -2/3;
* an independent construction through the HEALPix map projection of Calabretta &
  Roukema (2007): pixel centres form a regular lattice of diamonds in the
  projection plane, mapped back to the sphere with the projection's inverse;
* the equal-area property: the polar zone above ring i's centre holds exactly
  the pixels of rings 1..i-1 plus half of ring i.
"""
import math

import numpy as np
import pytest

import oracle


def test_base_resolution_centres():
    v = oracle.pix2vec_ring(1)
    z = v[:, 2]
    phi = np.mod(np.arctan2(v[:, 1], v[:, 0]), 2 * math.pi)
    np.testing.assert_allclose(z[:4], 2.0 / 3.0, atol=1e-15)
    np.testing.assert_allclose(z[4:8], 0.0, atol=1e-15)
    np.testing.assert_allclose(z[8:], -2.0 / 3.0, atol=1e-15)
    np.testing.assert_allclose(phi[:4], math.pi / 4 + np.arange(4) * math.pi / 2, atol=1e-14)
    np.testing.assert_allclose(phi[4:8], np.arange(4) * math.pi / 2, atol=1e-14)
    np.testing.assert_allclose(phi[8:], math.pi / 4 + np.arange(4) * math.pi / 2, atol=1e-14)


def _projection_centres(nside):
    """Pixel centres from the HEALPix projection plane (Calabretta & Roukema 2007).

    Returns (ring index k, z, phi) per pixel, unordered."""
    n = nside
    h = math.pi / (4 * n)
    facets = []
    for j in range(4):
        facets.append((math.pi / 4 + j * math.pi / 2, math.pi / 4))   # north
        facets.append((j * math.pi / 2, 0.0))                          # equatorial
        facets.append((math.pi / 4 + j * math.pi / 2, -math.pi / 4))  # south
    out = []
    u, v = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u = u.ravel()
    v = v.ravel()
    for x0, y0 in facets:
        x = x0 + (u - v) * h
        y = y0 - math.pi / 4 + (u + v + 1) * h
        k = np.rint((math.pi / 2 - y) / h).astype(np.int64)
        z = np.empty_like(y)
        phi = np.empty_like(y)
        eq = np.abs(y) <= math.pi / 4 + 1e-15
        z[eq] = 8.0 * y[eq] / (3.0 * math.pi)
        phi[eq] = x[eq]
        po = ~eq
        sg = 2.0 - 4.0 * np.abs(y[po]) / math.pi
        z[po] = np.sign(y[po]) * (1.0 - sg * sg / 3.0)
        xc = -math.pi + (2.0 * np.floor((x[po] + math.pi) * 2.0 / math.pi) + 1.0) * math.pi / 4
        phi[po] = xc + (x[po] - xc) / sg
        out.append((k, z, np.mod(phi, 2 * math.pi)))
    k = np.concatenate([o[0] for o in out])
    z = np.concatenate([o[1] for o in out])
    phi = np.concatenate([o[2] for o in out])
    # facet-edge lattice points are shared between neighbouring facets' grids only
    # at the boundaries, which the half-step offset keeps out; still dedupe safely.
    return k, z, phi


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16])
def test_projection_lattice_matches(nside):
    k, z, phi = _projection_centres(nside)
    assert len(k) == 12 * nside * nside
    order = np.lexsort((np.round(phi, 12), k))
    zc, pc = z[order], phi[order]
    v = oracle.pix2vec_ring(nside)
    zo = v[:, 2]
    po = np.mod(np.arctan2(v[:, 1], v[:, 0]), 2 * math.pi)
    np.testing.assert_allclose(zo, zc, atol=2e-15)
    d = np.abs(np.mod(po - pc + math.pi, 2 * math.pi) - math.pi)
    assert d.max() < 1e-12
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)


@pytest.mark.parametrize("nside", [2, 8, 64])
def test_equal_area_rings(nside):
    n = nside
    v = oracle.pix2vec_ring(n)
    z = v[:, 2]
    npix = 12 * n * n
    # ring boundaries in pixel order: z changes between rings
    starts = np.concatenate([[0], np.nonzero(np.diff(z))[0] + 1, [npix]])
    assert len(starts) - 1 == 4 * n - 1
    for r in range(4 * n - 1):
        a, b = starts[r], starts[r + 1]
        zr = z[a]
        if zr <= 0:
            continue
        area_above = 2 * math.pi * (1 - zr)  # spherical cap above the ring centre
        pixels_above = area_above * npix / (4 * math.pi)
        assert abs(pixels_above - (a + (b - a) / 2.0)) < 1e-6 * max(1.0, a)
