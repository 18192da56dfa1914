"""Pins of the oracle's Cartesian (projected) estimator, projS_pos (Sect. 2.2,
Sect. 5.2.1), and of its equal-area annulus statistics (Sect. 5.2.2).

  * the gnomonic projection against closed forms: the reference point maps
    to the origin, a point at angular distance rho maps to radius tan(rho)
    along its bearing, great circles map to straight lines, points more than
    90 degrees away have no image, and the printed trigonometric formula
    (Sect. 2.2.1) evaluated with numpy gives the same coordinates;
  * the shear rotation (Sect. 2.2.2): none for a reference point on the
    equator (projected meridians are parallel); otherwise the local North
    maps onto the direction of the image of the pole, (0, cot dec_c);
  * the estimator on a flat singular isothermal sphere: galaxies on a dense
    grid of the plane around a target, shear tangential in the plane and
    handed to the oracle in the local (East, North) basis, give
    M_E -> 4 theta_E / (5 theta_ap) (Schneider 1996, polynomial filter) and
    M_B = 0, which fixes the plane geometry, the sign of gamma_+, the
    rotation and the normalisation A = pi theta_ap^2;
  * a direct evaluation of Sect. 5.2.1's steps with trigonometry and atan2
    on tiny inputs; the 45-degree shear rotation; agreement with the
    spherical oracle near the reference point to O(theta_ap^2);
  * annuli: equal areas, and the mean / sd of a known difference pattern.
"""
import math

import numpy as np
import pytest

import oracle

ARCMIN = math.pi / (180 * 60)


def _vec(ra, dec):
    ra, dec = np.radians(ra), np.radians(dec)
    return np.stack([np.cos(dec) * np.cos(ra), np.cos(dec) * np.sin(ra), np.sin(dec)], -1)


def _offset(ra_c, dec_c, rho, bearing):
    """Points at angular distance rho and bearing (from North through East)
    from (ra_c, dec_c): spherical trigonometry, degrees in and out."""
    d0, a0 = math.radians(dec_c), math.radians(ra_c)
    sd = np.sin(d0) * np.cos(rho) + np.cos(d0) * np.sin(rho) * np.cos(bearing)
    dec = np.arcsin(sd)
    ra = a0 + np.arctan2(np.sin(bearing) * np.sin(rho) * np.cos(d0), np.cos(rho) - np.sin(d0) * sd)
    return np.degrees(ra), np.degrees(dec)


@pytest.mark.parametrize("ra_c,dec_c", [(30.0, 0.0), (200.0, 40.0), (300.0, -65.0)])
def test_projection_closed_forms(ra_c, dec_c):
    rng = np.random.default_rng(1)
    xy, ok = oracle.project(ra_c, dec_c, _vec([ra_c], [dec_c]))
    assert ok.all() and np.all(np.abs(xy) < 1e-15)
    rho = rng.uniform(1e-4, 1.2, 500)
    bear = rng.uniform(-math.pi, math.pi, 500)
    ra, dec = _offset(ra_c, dec_c, rho, bear)
    xy, ok = oracle.project(ra_c, dec_c, _vec(ra, dec))
    assert ok.all()
    np.testing.assert_allclose(np.hypot(xy[:, 0], xy[:, 1]), np.tan(rho), rtol=1e-12)
    # bearing from North (+y) through East (+x) is kept
    np.testing.assert_allclose(np.angle(np.exp(1j * (np.arctan2(xy[:, 0], xy[:, 1]) - bear))), 0, atol=1e-11)
    # beyond 90 degrees: no image
    ra, dec = _offset(ra_c, dec_c, rng.uniform(math.pi / 2 + 1e-6, math.pi - 1e-3, 50), rng.uniform(-3, 3, 50))
    _, ok = oracle.project(ra_c, dec_c, _vec(ra, dec))
    assert not ok.any()


def test_great_circles_map_to_lines():
    rng = np.random.default_rng(2)
    for _ in range(20):
        ra_c, dec_c = rng.uniform(0, 360), rng.uniform(-80, 80)
        # a great circle through two random points near the reference point
        c = _vec([ra_c], [dec_c])[0]
        a = c + rng.normal(0, 0.3, 3)
        b = c + rng.normal(0, 0.3, 3)
        a, b = a / np.linalg.norm(a), b / np.linalg.norm(b)
        t = rng.uniform(-0.5, 1.5, 30)
        pts = np.outer(1 - t, a) + np.outer(t, b)
        pts /= np.linalg.norm(pts, axis=1)[:, None]
        xy, ok = oracle.project(ra_c, dec_c, pts)
        assert ok.all()
        d = xy[1:] - xy[0]
        cross = d[1:, 0] * d[0, 1] - d[1:, 1] * d[0, 0]
        assert np.max(np.abs(cross)) < 1e-12 * max(1.0, np.max(np.abs(d)) ** 2)


def test_printed_projection_formula():
    # Sect. 2.2.1 as printed, with numpy trigonometry
    rng = np.random.default_rng(3)
    ra_c, dec_c = 123.0, -37.0
    ra, dec = _offset(ra_c, dec_c, rng.uniform(0, 0.6, 300), rng.uniform(-3, 3, 300))
    a, d, ac, dc = np.radians(ra), np.radians(dec), math.radians(ra_c), math.radians(dec_c)
    den = np.sin(d) * np.sin(dc) + np.cos(d) * np.cos(dc) * np.cos(a - ac)
    x = np.cos(d) * np.sin(a - ac) / den
    y = (np.cos(dc) * np.sin(d) - np.sin(dc) * np.cos(d) * np.cos(a - ac)) / den
    xy, ok = oracle.project(ra_c, dec_c, oracle.radec2vec(ra, dec))
    np.testing.assert_allclose(xy[:, 0], x, atol=1e-14)
    np.testing.assert_allclose(xy[:, 1], y, atol=1e-14)


def _pole_rotation(xy, dec_c):
    """Angle from +y (counter-clockwise) of the local North's image: towards
    the north pole's image (0, cot dec_c) for dec_c > 0, away from the south
    pole's image for dec_c < 0 (meridians are the lines through it)."""
    cot = 1.0 / math.tan(math.radians(dec_c))
    if dec_c > 0:
        return np.arctan2(xy[:, 0], cot - xy[:, 1])
    return np.arctan2(-xy[:, 0], xy[:, 1] - cot)


@pytest.mark.parametrize("dec_c", [0.0, 35.0, -55.0])
def test_shear_rotation_follows_local_north(dec_c):
    rng = np.random.default_rng(4)
    ra_c = 70.0
    ra, dec = _offset(ra_c, dec_c, rng.uniform(0, 0.5, 400), rng.uniform(-3, 3, 400))
    e1, e2 = rng.normal(0, 0.3, 400), rng.normal(0, 0.3, 400)
    g = oracle.plane_shear(ra_c, dec_c, ra, dec, e1, e2)
    if dec_c == 0.0:
        np.testing.assert_allclose(g[:, 0], e1, atol=1e-15)
        np.testing.assert_allclose(g[:, 1], e2, atol=1e-15)
        return
    xy, _ = oracle.project(ra_c, dec_c, oracle.radec2vec(ra, dec))
    want = (e1 + 1j * e2) * np.exp(2j * _pole_rotation(xy, dec_c))
    np.testing.assert_allclose(g[:, 0], want.real, atol=1e-13)
    np.testing.assert_allclose(g[:, 1], want.imag, atol=1e-13)


def _deproject(ra_c, dec_c, x, y):
    c = _vec([ra_c], [dec_c])[0]
    a, d = math.radians(ra_c), math.radians(dec_c)
    e = np.array([-math.sin(a), math.cos(a), 0.0])
    n = np.array([-math.sin(d) * math.cos(a), -math.sin(d) * math.sin(a), math.cos(d)])
    v = c[None, :] + x[:, None] * e[None, :] + y[:, None] * n[None, :]
    v /= np.linalg.norm(v, axis=1)[:, None]
    return np.degrees(np.arctan2(v[:, 1], v[:, 0])) % 360, np.degrees(np.arcsin(v[:, 2]))


@pytest.mark.parametrize("dec_c,x0,y0", [(40.0, 0.0, 0.0), (40.0, 0.05, -0.08), (-20.0, -0.1, 0.03)])
def test_flat_sis_closed_form(dec_c, x0, y0):
    ra_c, th, te = 15.0, 20 * ARCMIN, 0.5 * ARCMIN
    h = th / 300
    k = np.arange(-310, 311) * h
    gx, gy = np.meshgrid(k, k)
    gx, gy = gx.ravel() + x0 + 0.37 * h, gy.ravel() + y0 + 0.61 * h     # the target is not on the grid
    dx, dy = gx - x0, gy - y0
    r = np.hypot(dx, dy)
    phi = np.arctan2(dy, dx)
    gt = te / (2 * r)
    g_plane = -gt * np.exp(2j * phi)                 # tangential about the target, in the plane
    ra, dec = _deproject(ra_c, dec_c, gx, gy)
    xy, _ = oracle.project(ra_c, dec_c, oracle.radec2vec(ra, dec))
    rot = 0.0 if dec_c == 0 else _pole_rotation(xy, dec_c)
    g_loc = g_plane * np.exp(-2j * rot)              # handed over in the local (East, North) basis
    t_ra, t_dec = _deproject(ra_c, dec_c, np.array([x0]), np.array([y0]))
    cen = oracle.radec2vec(t_ra, t_dec)
    w = np.ones(gx.size)
    res = oracle.map_projected(cen, ra, dec, g_loc.real, g_loc.imag, w, ra_c, dec_c, 1, th)
    flat = 4 * te / (5 * th)
    assert res["ME"][0] == pytest.approx(flat, rel=2e-3)
    assert abs(res["MB"][0]) < 1e-9 * flat
    assert res["N"][0] == pytest.approx(math.pi * th * th / (h * h), rel=2e-3)


def _direct(c_ra, c_dec, ra_c, dec_c, ra, dec, e1, e2, w, kind, th):
    """Sect. 5.2.1 steps 1-4 with the printed projection, atan2 bearings and
    the pole-image rotation; plain loops over tiny inputs."""
    def proj(a_deg, d_deg):
        a, d, ac, dc = np.radians(a_deg), np.radians(d_deg), math.radians(ra_c), math.radians(dec_c)
        den = np.sin(d) * np.sin(dc) + np.cos(d) * np.cos(dc) * np.cos(a - ac)
        return (np.cos(d) * np.sin(a - ac) / den,
                (np.cos(dc) * np.sin(d) - np.sin(dc) * np.cos(d) * np.cos(a - ac)) / den)
    xi, yi = proj(ra, dec)
    rot = _pole_rotation(np.stack([xi, yi], -1), dec_c)
    g = (e1 + 1j * e2) * np.exp(2j * rot)
    out = []
    for a0, d0 in zip(c_ra, c_dec):
        x0, y0 = proj(np.array([a0]), np.array([d0]))
        dx, dy = xi - x0[0], yi - y0[0]
        r = np.hypot(dx, dy)
        m = r <= th
        phi = np.arctan2(dy[m], dx[m])
        q = oracle.filter_q(kind, r[m] / th) / th ** 2
        gp = -(g[m] * np.exp(-2j * phi)).real
        gxx = -(g[m] * np.exp(-2j * phi)).imag
        out.append((np.sum(w[m] * gp * q), np.sum(w[m] * gxx * q),
                    np.sum(w[m] ** 2 * np.abs(g[m]) ** 2 * q * q), np.sum(w[m]), m.sum()))
    return np.array(out)


@pytest.mark.parametrize("kind", [1, 2])
def test_direct_steps_tiny(kind):
    rng = np.random.default_rng(5)
    ra_c, dec_c, th = 250.0, 52.0, 25 * ARCMIN
    ra, dec = _offset(ra_c, dec_c, rng.uniform(0, 0.1, 800), rng.uniform(-3, 3, 800))
    e1, e2, w = rng.normal(0, 0.3, 800), rng.normal(0, 0.3, 800), rng.uniform(0.5, 1.5, 800)
    c_ra, c_dec = _offset(ra_c, dec_c, rng.uniform(0, 0.06, 12), rng.uniform(-3, 3, 12))
    ref = _direct(c_ra, c_dec, ra_c, dec_c, ra, dec, e1, e2, w, kind, th)
    got = oracle.aperture_projected(oracle.radec2vec(c_ra, c_dec), ra, dec, e1, e2, w, ra_c, dec_c, kind, th)
    np.testing.assert_array_equal(got["N"], ref[:, 4])
    sc = np.abs(ref[:, :2]).max()
    np.testing.assert_allclose(got["SE"], ref[:, 0], atol=1e-11 * sc)
    np.testing.assert_allclose(got["SB"], ref[:, 1], atol=1e-11 * sc)
    np.testing.assert_allclose(got["SV"], ref[:, 2], rtol=1e-11)
    np.testing.assert_allclose(got["SW"], ref[:, 3], rtol=1e-12)


def test_projected_shear_rotation_45():
    rng = np.random.default_rng(6)
    ra_c, dec_c, th = 10.0, -30.0, 30 * ARCMIN
    ra, dec = _offset(ra_c, dec_c, rng.uniform(0, 0.08, 3000), rng.uniform(-3, 3, 3000))
    e1, e2, w = rng.normal(0, 0.3, 3000), rng.normal(0, 0.3, 3000), rng.uniform(0.5, 1.5, 3000)
    cen = oracle.radec2vec(*_offset(ra_c, dec_c, rng.uniform(0, 0.05, 20), rng.uniform(-3, 3, 20)))
    a = oracle.map_projected(cen, ra, dec, e1, e2, w, ra_c, dec_c, 2, th)
    b = oracle.map_projected(cen, ra, dec, -e2, e1, w, ra_c, dec_c, 2, th)
    sc = np.abs(a["ME"]).max()
    np.testing.assert_allclose(b["ME"], -a["MB"], atol=1e-12 * sc)
    np.testing.assert_allclose(b["MB"], a["ME"], atol=1e-12 * sc)
    np.testing.assert_allclose(b["VAR"], a["VAR"], rtol=1e-12)


def test_agrees_with_spherical_near_the_reference_point():
    """At the reference point the plane is the sphere to second order: the
    projected and spherical sums of one target differ by O(theta_ap^2)."""
    rng = np.random.default_rng(7)
    ra_c, dec_c = 80.0, 25.0
    diffs = []
    n = 40000
    rad, bear = np.sqrt(rng.random(n)), rng.uniform(-3, 3, n)       # the same pattern at every scale
    e1, e2, w = rng.normal(0, 0.3, n), rng.normal(0, 0.3, n), np.ones(n)
    for th_arc in (4.0, 8.0, 16.0):
        th = th_arc * ARCMIN
        ra, dec = _offset(ra_c, dec_c, th * 1.05 * rad, bear)
        cen = oracle.radec2vec([ra_c], [dec_c])
        p = oracle.aperture_projected(cen, ra, dec, e1, e2, w, ra_c, dec_c, 1, th)
        s = oracle.aperture_galaxies(cen, ra, dec, e1, e2, w, 1, th)
        scale = np.sum(np.abs(w) * 6 / np.pi / th ** 2 * 0.25)
        diffs.append(max(abs(p["SE"][0] - s["SE"][0]), abs(p["SB"][0] - s["SB"][0])) / scale)
    assert diffs[-1] < 2e-4
    # quadratic in theta_ap: doubling the aperture multiplies the difference by about 4
    assert 2.0 < diffs[2] / diffs[1] < 8.0 and 2.0 < diffs[1] / diffs[0] < 8.0


def test_annuli_have_equal_area_and_known_statistics():
    nside = 256
    ref = oracle.radec2vec([0.0], [0.0])[0]
    v = oracle.pix2vec(nside, np.arange(12 * nside * nside))
    rmax = math.radians(20.0)
    cosd = v @ ref
    sel = cosd > math.cos(rmax)
    v = v[sel]
    nb = 10
    rng = np.random.default_rng(8)
    mref = rng.normal(0, 2.0, len(v))
    u = 1 - v @ ref
    k = np.minimum((u / (1 - math.cos(rmax)) * nb).astype(int), nb - 1)
    # annulus k: a constant offset a_k on even annuli, +-b_k on odd ones
    a = 0.1 * np.arange(nb)
    sign = np.where(rng.random(len(v)) < 0.5, -1.0, 1.0)
    mx = mref + np.where(k % 2 == 0, a[k], a[k] * sign)
    st = oracle.annulus_stats(v, ref, rmax, mx, mref, nb)
    sref = np.std(mref)
    # equal areas: HEALPix pixels have equal area, so the counts agree to the
    # pixel-boundary noise of each annulus
    assert st["count"].sum() == len(v)
    np.testing.assert_allclose(st["count"], len(v) / nb, rtol=0.03)
    even = np.arange(0, nb, 2)
    np.testing.assert_allclose(st["mean"][even], a[even] / sref, atol=1e-12)
    np.testing.assert_allclose(st["sd"][even], 0.0, atol=1e-6)
    odd = np.arange(1, nb, 2)
    np.testing.assert_allclose(st["sd"][odd], a[odd] / sref, rtol=0.02)
