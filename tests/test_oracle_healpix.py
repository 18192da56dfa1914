"""Pins of the oracle's elementary functions and HEALPix RING geometry.

The HEALPix grid (Gorski et al. 2005, cited in Sect. 3 of the paper) is
pinned by its defining properties: pixel counts per ring, ring latitudes,
equal pixel areas, the 90-degree and north-south symmetries of the grid,
and exhaustive centre -> pixel round trips.  The series sine/cosine is
pinned against 50-digit mpmath.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle

mpmath.mp.dps = 50


def _ulp(x):
    return np.spacing(abs(x)) if x != 0 else np.spacing(0.0)


@pytest.mark.parametrize("unit", ["deg", "quarter"])
def test_sincos_against_mpmath(unit):
    rng = np.random.default_rng(7)
    xs = np.concatenate([rng.uniform(-1000, 1000, 1500), rng.uniform(-1, 1, 300),
                         np.array([0.0, 45.0, 90.0, 135.0, -45.0, 1e-300, 89.999999999, 360.0])])
    for x in xs:
        if unit == "deg":
            s, c = oracle.sincos_deg(x)
            ang = mpmath.mpf(x) * mpmath.pi / 180
        else:
            s, c = oracle.sincos_quarter(x)
            ang = mpmath.mpf(x) * mpmath.pi / 2
        se, ce = float(mpmath.sin(ang)), float(mpmath.cos(ang))
        # within 2 ulp of the magnitude-1 scale, and relative for tiny values
        assert abs(s - se) <= max(2 * _ulp(se), 4e-16 * abs(se), 2.3e-16 if abs(se) > 1e-3 else 1e-300) + 3e-17, (x, s, se)
        assert abs(c - ce) <= max(2 * _ulp(ce), 4e-16 * abs(ce), 2.3e-16 if abs(ce) > 1e-3 else 1e-300) + 3e-17, (x, c, ce)


def test_sincos_tiny_relative():
    for x in [1e-10, 3e-7, -2e-5, 1e-3]:
        s, _ = oracle.sincos_deg(x)
        exact = float(mpmath.sin(mpmath.mpf(x) * mpmath.pi / 180))
        assert abs(s - exact) <= 2 * _ulp(exact)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 64])
def test_ring_structure(nside):
    N = nside
    total = 0
    for i in range(1, 4 * N):
        start, nr, z, sh = oracle.ring_info(N, i)
        assert start == total
        total += nr
        if i < N:
            assert nr == 4 * i and z == pytest.approx(1 - i * i / (3 * N * N), abs=1e-15)
        elif i <= 3 * N:
            assert nr == 4 * N and z == pytest.approx(4 / 3 - 2 * i / (3 * N), abs=1e-15)
        else:
            s = 4 * N - i
            assert nr == 4 * s and z == pytest.approx(-(1 - s * s / (3 * N * N)), abs=1e-15)
    assert total == 12 * N * N


def test_nside1_centres():
    # the twelve base pixels: three rings of four at z = 2/3, 0, -2/3
    v = oracle.pix2vec(1, np.arange(12))
    z = v[:, 2]
    phi = np.degrees(np.arctan2(v[:, 1], v[:, 0])) % 360
    np.testing.assert_allclose(z, [2 / 3] * 4 + [0] * 4 + [-2 / 3] * 4, atol=1e-15)
    np.testing.assert_allclose(phi, [45, 135, 225, 315, 0, 90, 180, 270, 45, 135, 225, 315], atol=1e-12)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 32, 64])
def test_centre_roundtrip_exhaustive(nside):
    npix = 12 * nside * nside
    pix = np.arange(npix)
    v = oracle.pix2vec(nside, pix)
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=4e-16)
    ra = np.degrees(np.arctan2(v[:, 1], v[:, 0])) % 360
    dec = np.degrees(np.arcsin(np.clip(v[:, 2], -1, 1)))
    back = oracle.ang2pix(nside, ra, dec)
    np.testing.assert_array_equal(back, pix)


def test_pix_info_consistency():
    for nside in (4, 16):
        for p in range(12 * nside * nside):
            ring, j, nr, z, rho, f = oracle.pix_info(nside, p)
            start, nr2, z2, sh = oracle.ring_info(nside, ring)
            assert start + j == p and nr2 == nr and z2 == z
            assert abs(rho * rho + z * z - 1) < 4e-16
            # phi in quarter turns: (j + 1/2) / (nr/4) on shifted rings, j / (nr/4) otherwise
            assert f == pytest.approx((j + (0.5 if sh else 0.0)) / (nr / 4), rel=0, abs=1e-14)


@pytest.mark.parametrize("nside", [2, 4])
def test_equal_area(nside):
    # uniform points on the sphere fall into every pixel with equal probability
    rng = np.random.default_rng(11)
    n = 2_000_000
    z = rng.uniform(-1, 1, n)
    ra = rng.uniform(0, 360, n)
    dec = np.degrees(np.arcsin(z))
    pix = oracle.ang2pix(nside, ra, dec)
    npix = 12 * nside * nside
    counts = np.bincount(pix, minlength=npix)
    exp = n / npix
    chi2 = np.sum((counts - exp) ** 2 / exp)
    # chi^2 with npix-1 dof: mean npix-1, sd sqrt(2(npix-1))
    assert chi2 < npix - 1 + 6 * math.sqrt(2 * (npix - 1)), chi2


@pytest.mark.parametrize("nside", [1, 8, 128, 4096])
def test_grid_symmetries(nside):
    rng = np.random.default_rng(3)
    n = 20000
    ra = rng.uniform(0, 360, n)
    dec = np.degrees(np.arcsin(rng.uniform(-1, 1, n)))
    p = oracle.ang2pix(nside, ra, dec)
    p90 = oracle.ang2pix(nside, (ra + 90.0) % 360, dec)
    pm = oracle.ang2pix(nside, ra, -dec)
    for a, b, c in zip(p[:3000], p90[:3000], pm[:3000]):
        ring, j, nr, *_ = oracle.pix_info(nside, int(a))
        r2, j2, nr2, *_ = oracle.pix_info(nside, int(b))
        assert r2 == ring and j2 == (j + nr // 4) % nr
        r3, j3, nr3, *_ = oracle.pix_info(nside, int(c))
        assert r3 == 4 * nside - ring and j3 == j


def test_random_points_near_centre():
    # a point close to a centre (well inside the pixel) maps to that pixel
    rng = np.random.default_rng(5)
    nside = 4096
    pix = rng.integers(0, 12 * nside * nside, 5000)
    v = oracle.pix2vec(nside, pix)
    eps = 0.05 * math.sqrt(4 * math.pi / (12 * nside * nside))
    d = rng.normal(size=v.shape)
    d -= (d * v).sum(1)[:, None] * v
    d /= np.linalg.norm(d, axis=1)[:, None]
    q = v + eps * d
    q /= np.linalg.norm(q, axis=1)[:, None]
    ra = np.degrees(np.arctan2(q[:, 1], q[:, 0])) % 360
    dec = np.degrees(np.arcsin(q[:, 2]))
    np.testing.assert_array_equal(oracle.ang2pix(nside, ra, dec), pix)


def test_poles_and_wrap():
    for nside in (1, 2, 64, 4096):
        assert oracle.ang2pix(nside, 10.0, 90.0) in range(4)
        assert oracle.ang2pix(nside, 10.0, -90.0) in range(12 * nside * nside - 4, 12 * nside * nside)
        assert oracle.ang2pix(nside, 360.0, 0.3) == oracle.ang2pix(nside, 0.0, 0.3)
        assert oracle.ang2pix(nside, -90.0, 12.0) == oracle.ang2pix(nside, 270.0, 12.0)


@pytest.mark.parametrize("nside", [4, 8, 32])
def test_query_disc_matches_all_pixels(nside):
    rng = np.random.default_rng(nside)
    cases = []
    for _ in range(40):
        zc = rng.uniform(-1, 1)
        ph = rng.uniform(0, 2 * math.pi)
        r = math.sqrt(1 - zc * zc)
        cases.append((np.array([r * math.cos(ph), r * math.sin(ph), zc]), rng.uniform(0.01, 0.6)))
    cases.append((np.array([0.0, 0.0, 1.0]), 0.3))       # north pole
    cases.append((np.array([0.0, 0.0, -1.0]), 0.2))      # south pole
    cases.append((np.array([1.0, 0.0, 0.0]), 3.0))       # nearly whole sky
    cases.append((oracle.pix2vec(nside, [5])[0], 1e-9))  # tiny disc at a centre
    for r0, th in cases:
        a = oracle.query_disc(nside, r0, th)
        b = oracle.query_disc(nside, r0, th, all_pixels=True)
        np.testing.assert_array_equal(np.sort(a), b)


def test_pixel_sizes_printed_in_the_paper():
    """The angular pixel sizes the paper prints for NSIDE 2048 to 16384
    (tests/golden/pixel_sizes.json, with its citation) follow from the
    oracle's ring structure: the pixel count (first pixel of the last ring
    plus its length) divides the full sphere into equal areas."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pixel_sizes.json")))
    for nside, printed in zip(g["nside"], g["pixel_size_arcmin"]):
        first, count, _, _ = oracle.ring_info(nside, 4 * nside - 1)
        npix = first + count
        size = math.degrees(math.sqrt(4.0 * math.pi / npix)) * 60.0
        assert round(size, 2) == printed, (nside, size, printed)

