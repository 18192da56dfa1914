"""Pins of the oracle's aperture sums against closed forms, invariants and an
independent evaluation of the paper's printed spherical formulas.

  * filter: Q from U (Sect. 2), compensation of U, Schirmer limits;
  * a direct O(N M) evaluation of Sect. 2.3's separation and tan(psi)
    formulas with atan2 (not unit vectors) on tiny inputs;
  * the isolated SIS: M_B = 0 and M_E = integral of Q gamma_t over the cap
    (1-D quadrature), tending to 4 theta_E / (5 theta_ap) in the flat limit;
  * invariants: 45-degree shear rotation, RA shift by 90 degrees, N-S
    mirror, a general rigid rotation, constant shear;
  * the flat-sky limit: gnomonic-plane estimator on the equator, O(theta_ap^2);
  * pixel mode equals brute force on the catalogue snapped to pixel centres;
  * binning equals numpy's stable argsort / bincount;
  * the noise map (Eq. 8) equals the Monte Carlo variance of M_E and M_B
    under pure shape noise.
"""
import math

import numpy as np
import pytest
import torch
from scipy import integrate

import oracle
from paper_2609_11181_b300 import synth

ARCMIN = math.pi / (180 * 60)


# ------------------------------------------------------------------ filters
def test_q_from_u_poly():
    # Q(x) = (2/x^2) int_0^x x' U(x') dx' - U(x)   (Sect. 2, Q from U)
    for x in [0.05, 0.2, 0.5, 0.77, 0.99]:
        integral, _ = integrate.quad(lambda t: t * oracle.filter_u_poly(t)[0], 0, x,
                                     epsabs=1e-14, epsrel=1e-13)
        q = 2 / x ** 2 * integral - oracle.filter_u_poly(x)[0]
        assert q == pytest.approx(oracle.filter_q(1, x)[0], rel=1e-11, abs=1e-14)


def test_u_compensated():
    x, wx = np.polynomial.legendre.leggauss(8)      # exact for this degree-5 integrand
    t = 0.5 * (x + 1)
    val = 0.5 * np.sum(wx * t * oracle.filter_u_poly(t))
    assert abs(val) < 1e-14


def test_schirmer_limits():
    xc = 0.15
    q0 = oracle.filter_q(2, 1e-12, xc)[0]
    assert q0 == pytest.approx(1 / (1 + math.exp(6) + math.exp(-47)), rel=1e-9)
    # away from both exponential cut-offs the filter is tanh(x/xc)/(x/xc)
    x = 0.5
    assert oracle.filter_q(2, x, xc)[0] == pytest.approx(math.tanh(x / xc) / (x / xc), rel=1e-8)
    # the outer cut-off halves the filter where -47 + 50 x = 0
    x = 0.94
    assert oracle.filter_q(2, x, xc)[0] == pytest.approx(0.5 * math.tanh(x / xc) / (x / xc), rel=1e-6)


# ---------------------------------------------- direct spherical formulas
def _direct(c_ra, c_dec, ra, dec, e1, e2, w, kind, theta_ap):
    """Sect. 2.3's printed formulas, evaluated with trig + atan2."""
    a0, d0 = np.radians(c_ra), np.radians(c_dec)
    ai, di = np.radians(ra), np.radians(dec)
    out = []
    for a, d in zip(a0, d0):
        da = ai - a
        cosd = np.sin(di) * np.sin(d) + np.cos(di) * np.cos(d) * np.cos(da)
        # haversine for an accurate separation at small angles
        hav = np.sin((di - d) / 2) ** 2 + np.cos(di) * np.cos(d) * np.sin(da / 2) ** 2
        sep = 2 * np.arcsin(np.sqrt(hav))
        assert np.allclose(np.cos(sep), cosd, atol=1e-12)
        m = sep <= theta_ap
        psi = np.arctan2(np.sin(da), np.cos(di) * np.tan(d) - np.sin(di) * np.cos(da))
        q = oracle.filter_q(kind, sep[m] / theta_ap) / theta_ap ** 2
        gp = e1[m] * np.cos(2 * psi[m]) + e2[m] * np.sin(2 * psi[m])
        gx = -e1[m] * np.sin(2 * psi[m]) + e2[m] * np.cos(2 * psi[m])
        out.append((np.sum(w[m] * gp * q), np.sum(w[m] * gx * q),
                    np.sum(w[m] ** 2 * (e1[m] ** 2 + e2[m] ** 2) * q * q), np.sum(w[m]), m.sum()))
    return np.array(out)


@pytest.mark.parametrize("kind", [1, 2])
def test_direct_formulas_tiny(kind):
    rng = np.random.default_rng(kind)
    n, n0 = 600, 40
    ra = rng.uniform(20, 26, n)
    dec = rng.uniform(-33, -27, n)
    e1, e2 = rng.normal(0, 0.3, n), rng.normal(0, 0.3, n)
    w = rng.uniform(0.5, 1.5, n)
    c_ra, c_dec = rng.uniform(21, 25, n0), rng.uniform(-32, -28, n0)
    th = 1.5 * math.pi / 180
    ref = _direct(c_ra, c_dec, ra, dec, e1, e2, w, kind, th)
    cv = oracle.radec2vec(c_ra, c_dec)
    got = oracle.aperture_galaxies(cv, ra, dec, e1, e2, w, kind, th)
    np.testing.assert_array_equal(got["N"], ref[:, 4].astype(np.int64))
    for k, col in (("SE", 0), ("SB", 1), ("SV", 2), ("SW", 3)):
        np.testing.assert_allclose(got[k], ref[:, col], rtol=1e-10, atol=1e-10 * np.abs(ref[:, col]).max())


# --------------------------------------------------------------- SIS pin
def _polar_grid(ra0, dec0, theta_max, n_t=64, n_p=160):
    """Gauss-Legendre nodes in theta x uniform phi around (ra0, dec0); weights = dOmega."""
    x, wx = np.polynomial.legendre.leggauss(n_t)
    th = 0.5 * theta_max * (x + 1)
    wt = 0.5 * theta_max * wx * np.sin(th)
    ph = (np.arange(n_p) + 0.5) * 2 * np.pi / n_p
    T, P = np.meshgrid(th, ph, indexing="ij")
    W = np.repeat(wt[:, None], n_p, axis=1) * (2 * np.pi / n_p)
    v = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    # rotate +z onto (ra0, dec0)
    t = math.pi / 2 - math.radians(dec0)
    Ry = np.array([[math.cos(t), 0, math.sin(t)], [0, 1, 0], [-math.sin(t), 0, math.cos(t)]])
    a = math.radians(ra0)
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    v = v @ (Rz @ Ry).T
    ra = np.degrees(np.arctan2(v[:, 1], v[:, 0])) % 360
    dec = np.degrees(np.arcsin(np.clip(v[:, 2], -1, 1)))
    return ra, dec, W.ravel()


@pytest.mark.parametrize("kind,theta_arcmin,dec0", [(1, 60, 24.0), (1, 10, -61.0), (2, 10, 5.0), (1, 600, 40.0)])
def test_sis_closed_form(kind, theta_arcmin, dec0):
    th = theta_arcmin * ARCMIN
    te = 0.7 * ARCMIN
    ra0 = 37.0
    ra, dec, w = _polar_grid(ra0, dec0, th * (1 - 1e-9), n_t=400 if kind == 2 else 64)
    halos = synth.Halos(torch.tensor([ra0], dtype=torch.float64), torch.tensor([dec0], dtype=torch.float64),
                        torch.tensor([te], dtype=torch.float64))
    g1, g2 = synth.sis_shear(torch.from_numpy(ra), torch.from_numpy(dec), halos, r_trunc=2 * th, inner_cut=False)
    e1, e2 = g1.numpy(), g2.numpy()
    c = oracle.radec2vec([ra0], [dec0])
    r = oracle.map_galaxies(c, ra, dec, e1, e2, w, kind, th)

    def integrand(t):
        return 2 * math.pi * math.sin(t) * oracle.filter_q(kind, t / th)[0] / th ** 2 * te / (2 * t)

    exact, _ = integrate.quad(integrand, 0, th, epsabs=1e-15, epsrel=1e-12, limit=200)
    assert r["SW"][0] == pytest.approx(2 * math.pi * (1 - math.cos(th * (1 - 1e-9))), rel=1e-12)
    assert r["ME"][0] == pytest.approx(exact, rel=1e-8)
    assert abs(r["MB"][0]) < 1e-11 * abs(exact)
    if kind == 1 and theta_arcmin <= 60:
        flat = 4 * te / (5 * th)          # Schneider (1996) flat-sky closed form
        assert r["ME"][0] == pytest.approx(flat, rel=2 * th ** 2)


# ---------------------------------------------------------- invariants
def _catalog(seed, n=4000, ra0=30.0, dec0=10.0, radius_deg=3.0, nhalo=6):
    g = synth.make_gen(seed)
    rad = math.radians(radius_deg)
    halos = synth.halos_uniform(nhalo, ra0, dec0, rad, g, 0.2 * ARCMIN, 1.0 * ARCMIN)
    cat = synth.galaxy_catalog(n, ra0, dec0, rad, halos, g, r_trunc=math.radians(2.0), w_range=(0.5, 1.5))
    return (cat.ra_deg.numpy(), cat.dec_deg.numpy(), cat.e1.double().numpy(),
            cat.e2.double().numpy(), cat.w.double().numpy())


def _targets(nside, ra0, dec0, radius_deg):
    v = oracle.pix2vec(nside, np.arange(12 * nside * nside))
    c = oracle.radec2vec([ra0], [dec0])[0]
    return np.nonzero(v @ c >= math.cos(math.radians(radius_deg)))[0]


def test_shear_rotation_45():
    ra, dec, e1, e2, w = _catalog(1)
    tg = _targets(64, 30, 10, 2.0)
    cv = oracle.pix2vec(64, tg)
    th = 30 * ARCMIN
    a = oracle.map_galaxies(cv, ra, dec, e1, e2, w, 1, th)
    b = oracle.map_galaxies(cv, ra, dec, -e2, e1, w, 1, th)
    sc = np.abs(a["ME"]).max()
    np.testing.assert_allclose(b["ME"], -a["MB"], atol=1e-12 * sc)
    np.testing.assert_allclose(b["MB"], a["ME"], atol=1e-12 * sc)
    np.testing.assert_allclose(b["VAR"], a["VAR"], rtol=1e-12)


def test_ra_shift_90_permutes_map():
    nside = 64
    ra, dec, e1, e2, w = _catalog(2)
    tg = _targets(nside, 30, 10, 2.0)
    th = 25 * ARCMIN
    a = oracle.map_galaxies(oracle.pix2vec(nside, tg), ra, dec, e1, e2, w, 2, th)
    tg2 = []
    for p in tg:
        ring, j, nr, *_ = oracle.pix_info(nside, int(p))
        start, *_ = oracle.ring_info(nside, ring)
        tg2.append(start + (j + nr // 4) % nr)
    b = oracle.map_galaxies(oracle.pix2vec(nside, np.array(tg2)), (ra + 90.0) % 360, dec, e1, e2, w, 2, th)
    np.testing.assert_array_equal(a["N"], b["N"])
    sc = np.abs(a["ME"]).max()
    np.testing.assert_allclose(b["ME"], a["ME"], atol=1e-10 * sc)
    np.testing.assert_allclose(b["MB"], a["MB"], atol=1e-10 * sc)


def test_north_south_mirror():
    nside = 64
    ra, dec, e1, e2, w = _catalog(3)
    tg = _targets(nside, 30, 10, 2.0)
    th = 25 * ARCMIN
    a = oracle.map_galaxies(oracle.pix2vec(nside, tg), ra, dec, e1, e2, w, 1, th)
    tm = []
    for p in tg:
        ring, j, *_ = oracle.pix_info(nside, int(p))
        start, *_ = oracle.ring_info(nside, 4 * nside - ring)
        tm.append(start + j)
    b = oracle.map_galaxies(oracle.pix2vec(nside, np.array(tm)), ra, -dec, e1, -e2, w, 1, th)
    np.testing.assert_array_equal(a["N"], b["N"])
    sc = np.abs(a["ME"]).max()
    np.testing.assert_allclose(b["ME"], a["ME"], atol=1e-10 * sc)
    np.testing.assert_allclose(b["MB"], -a["MB"], atol=1e-10 * sc)


def _basis(v):
    rho = np.hypot(v[:, 0], v[:, 1])
    e = np.stack([-v[:, 1] / rho, v[:, 0] / rho, np.zeros(len(v))], -1)
    nn = np.stack([-v[:, 2] * v[:, 0] / rho, -v[:, 2] * v[:, 1] / rho, rho], -1)
    return e, nn


def test_rigid_rotation():
    ra, dec, e1, e2, w = _catalog(4, n=3000)
    v = oracle.radec2vec(ra, dec)
    rng = np.random.default_rng(9)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    R = q
    vr = v @ R.T
    ea, na = _basis(v)
    eb, nb = _basis(vr)
    Re = ea @ R.T
    chi = np.arctan2((nb * Re).sum(1), (eb * Re).sum(1))      # old East seen in the new basis
    g = (e1 + 1j * e2) * np.exp(2j * chi)
    ra2 = np.degrees(np.arctan2(vr[:, 1], vr[:, 0])) % 360
    dec2 = np.degrees(np.arcsin(np.clip(vr[:, 2], -1, 1)))
    cen = oracle.radec2vec(rng.uniform(28.5, 31.5, 30), rng.uniform(8.5, 11.5, 30))
    th = 40 * ARCMIN
    a = oracle.map_galaxies(cen, ra, dec, e1, e2, w, 1, th)
    b = oracle.map_galaxies(cen @ R.T, ra2, dec2, g.real, g.imag, w, 1, th)
    np.testing.assert_array_equal(a["N"], b["N"])
    sc = np.abs(a["ME"]).max()
    np.testing.assert_allclose(b["ME"], a["ME"], atol=1e-9 * sc)
    np.testing.assert_allclose(b["MB"], a["MB"], atol=1e-9 * sc)


def _flat_sky_difference(theta_arcmin, n=20000, seed=5):
    """|S_flat - S_oracle| / (0.05 sum |w Q|) for E and B at one centre on the
    equator.  The flat estimator (Sect. 2.2: the galaxies' positions in the
    tangent plane by gnomonic projection) takes those coordinates about the centre,
    the bearing from atan2 in that plane and the polynomial filter of the
    projected distance; it shares nothing with the oracle's code.  On the
    equator the galaxies' local (East, North) bases differ from the projected
    axes only at second order, so every difference is O(theta_ap^2)."""
    th = theta_arcmin * ARCMIN
    rng = np.random.default_rng(seed)
    r = 1.2 * th * np.sqrt(rng.random(n))
    a = 2 * math.pi * rng.random(n)
    a0 = math.radians(40.0)
    c0 = np.array([math.cos(a0), math.sin(a0), 0.0])
    east, north = np.array([-math.sin(a0), math.cos(a0), 0.0]), np.array([0.0, 0.0, 1.0])
    xi1, xi2 = r * np.cos(a), r * np.sin(a)
    v = c0[None, :] + xi1[:, None] * east[None, :] + xi2[:, None] * north[None, :]
    v /= np.linalg.norm(v, axis=1)[:, None]
    dec = np.degrees(np.arcsin(v[:, 2]))
    ra = np.degrees(np.arctan2(v[:, 1], v[:, 0])) % 360
    phi = np.arctan2(xi2, xi1)
    e1 = -0.05 * np.cos(2 * phi) + 0.02 * rng.standard_normal(n)   # tangential field + noise
    e2 = -0.05 * np.sin(2 * phi) + 0.02 * rng.standard_normal(n)
    w = 0.5 + rng.random(n)
    s = oracle.aperture_galaxies(c0[None, :], ra, dec, e1, e2, w, 1, th)
    cosd = v @ c0
    p1, p2 = (v @ east) / cosd, (v @ north) / cosd
    x = np.hypot(p1, p2) / th
    f = np.arctan2(p2, p1)
    m = x <= 1.0
    q = 6 / math.pi * x ** 2 * (1 - x ** 2) / th ** 2
    gt = -(e1 * np.cos(2 * f) + e2 * np.sin(2 * f))
    gx = e1 * np.sin(2 * f) - e2 * np.cos(2 * f)
    scale = 0.05 * np.sum(np.abs(w * q)[m])
    assert int(m.sum()) == int(s["N"][0])
    return (abs(np.sum((w * gt * q)[m]) - s["SE"][0]) / scale,
            abs(np.sum((w * gx * q)[m]) - s["SB"][0]) / scale)


def test_flat_sky_limit():
    # Sect. 2.3's spherical estimator reduces to Sect. 2.2's flat one as theta_ap -> 0,
    # with differences of order theta_ap^2 (measured: 0.66 theta_ap^2 for E)
    d = {t: _flat_sky_difference(t) for t in (1.0, 4.0, 16.0)}
    for t, (de, db) in d.items():
        th2 = (t * ARCMIN) ** 2
        assert de < th2 and db < th2, (t, de, db, th2)
    for lo, hi in ((1.0, 4.0), (4.0, 16.0)):
        assert 12.0 < d[hi][0] / d[lo][0] < 20.0, d     # quadratic: x16 for 4x theta_ap


def test_constant_shear_vanishes():
    # on a polar grid about an equatorial centre, a shear constant in the local
    # basis averages out over azimuth; what is left is the O(theta^2) turn of
    # the local basis across the aperture
    th = 20 * ARCMIN
    ra, dec, w = _polar_grid(123.0, 0.0, th * (1 - 1e-9))
    e1 = np.full(ra.size, 0.1)
    e2 = np.full(ra.size, -0.05)
    r = oracle.map_galaxies(oracle.radec2vec([123.0], [0.0]), ra, dec, e1, e2, w, 1, th)
    assert abs(r["ME"][0]) < 0.1 * th ** 2 and abs(r["MB"][0]) < 0.1 * th ** 2


# --------------------------------------------- pixel mode and binning
def test_binning_against_numpy():
    ra, dec, e1, e2, w = _catalog(5, n=20000)
    nside = 256
    b = oracle.bin_catalog(nside, ra, dec, e1, e2, w)
    pix = oracle.ang2pix(nside, ra, dec)
    np.testing.assert_array_equal(b["pix"], pix)
    np.testing.assert_array_equal(b["perm"], np.argsort(pix, kind="stable"))
    npix = 12 * nside * nside
    cnt = np.bincount(pix, minlength=npix)
    np.testing.assert_array_equal(b["n"], cnt)
    np.testing.assert_array_equal(b["offsets"], np.concatenate([[0], np.cumsum(cnt)]))
    np.testing.assert_allclose(b["G1"], np.bincount(pix, w * e1, npix), atol=1e-12)
    np.testing.assert_allclose(b["S2"], np.bincount(pix, w * w * (e1 ** 2 + e2 ** 2), npix), atol=1e-12)


@pytest.mark.parametrize("kind", [1, 2])
def test_pixel_mode_equals_snapped_brute_force(kind):
    ra, dec, e1, e2, w = _catalog(6, n=30000)
    nb, no = 256, 64
    b = oracle.bin_catalog(nb, ra, dec, e1, e2, w)
    pv = oracle.pix2vec(nb, b["pix"])
    sra = np.degrees(np.arctan2(pv[:, 1], pv[:, 0])) % 360
    sdec = np.degrees(np.arcsin(np.clip(pv[:, 2], -1, 1)))
    tg = _targets(no, 30, 10, 2.2)
    cv = oracle.pix2vec(no, tg)
    th = 35 * ARCMIN
    a = oracle.map_pixels(cv, nb, b["G1"], b["G2"], b["W"], b["S2"], b["n"], kind, th)
    s = oracle.map_galaxies(cv, sra, sdec, e1, e2, w, kind, th)
    np.testing.assert_array_equal(a["N"], s["N"])
    for k in ("SE", "SB", "SV", "SW"):
        np.testing.assert_allclose(a[k], s[k], rtol=1e-9, atol=1e-9 * np.abs(s[k]).max())


@pytest.mark.parametrize("kind", [1, 2])
def test_own_pixel_carries_no_shear(kind):
    # a binned map whose only non-empty pixel is the target's own pixel: the
    # position angle is undefined at the centre, so M_E = M_B = 0 exactly,
    # while the weight and the noise term still count
    nside = 256
    npix = 12 * nside * nside
    rng = np.random.default_rng(kind)
    for p in rng.integers(0, npix, 25):
        G1, G2, W, S2 = (np.zeros(npix) for _ in range(4))
        n = np.zeros(npix, dtype=np.int64)
        G1[p], G2[p], W[p], S2[p], n[p] = 3.0, -2.0, 5.0, 0.7, 5
        r = oracle.map_pixels(oracle.pix2vec(nside, [p]), nside, G1, G2, W, S2, n, kind, 20 * ARCMIN)
        assert r["SE"][0] == 0.0 and r["SB"][0] == 0.0
        assert r["SW"][0] == 5.0 and r["N"][0] == 5
        q0 = oracle.filter_q(kind, 0.0)[0] / (20 * ARCMIN) ** 2
        assert r["SV"][0] == pytest.approx(q0 * q0 * 0.7, rel=1e-12, abs=1e-300)


# --------------------------------------------------------------------------
# barycentre form of the pixel-based map (Sect. 3.3)
# --------------------------------------------------------------------------
def _spread_catalog(seed, nside, ra0, dec0, rad_deg, per_pixel_max_one=True, n=3000):
    """Galaxies at most one per pixel (drawn pixel by pixel inside a cap)."""
    rng = np.random.default_rng(seed)
    v = oracle.pix2vec(nside, np.arange(12 * nside * nside))
    c = oracle.radec2vec([ra0], [dec0])[0]
    pix = np.nonzero(v @ c >= np.cos(np.radians(rad_deg)))[0]
    pick = rng.choice(pix, size=min(n, pix.size), replace=False)
    # a point near each picked centre, well inside its pixel
    pv = v[pick] + rng.normal(0, 0.05 * np.sqrt(4 * np.pi / (12 * nside * nside)), (pick.size, 3))
    pv /= np.linalg.norm(pv, axis=1)[:, None]
    ra = np.degrees(np.arctan2(pv[:, 1], pv[:, 0])) % 360.0
    dec = np.degrees(np.arcsin(np.clip(pv[:, 2], -1, 1)))
    keep = oracle.ang2pix(nside, ra, dec) == pick
    ra, dec = ra[keep], dec[keep]
    e1 = rng.normal(0, 0.26, ra.size)
    e2 = rng.normal(0, 0.26, ra.size)
    w = rng.uniform(0.5, 1.5, ra.size)
    return ra, dec, e1, e2, w


def test_barycentre_map_equals_brute_force_with_one_galaxy_per_pixel():
    nside = 256
    ra, dec, e1, e2, w = _spread_catalog(11, nside, 30.0, 20.0, 3.0)
    assert np.bincount(oracle.ang2pix(nside, ra, dec)).max() == 1
    tg = oracle.pix2vec(64, np.arange(12 * 64 * 64))
    c = oracle.radec2vec([30.0], [20.0])[0]
    tg = tg[tg @ c >= np.cos(np.radians(1.5))]
    th = 40.0 * ARCMIN
    bf = oracle.map_galaxies(tg, ra, dec, e1, e2, w, 2, th)
    pb = oracle.map_barycentre(tg, nside, ra, dec, e1, e2, w, 2, th)
    np.testing.assert_array_equal(pb["N"], bf["N"])
    np.testing.assert_array_equal(pb["K"], bf["N"])
    for k in ("ME", "MB", "VAR", "SW"):
        np.testing.assert_allclose(pb[k], bf[k], rtol=1e-10, atol=1e-14)


def test_barycentre_map_equals_pixel_map_when_galaxies_sit_at_centres():
    nside = 128
    rng = np.random.default_rng(12)
    v = oracle.pix2vec(nside, np.arange(12 * nside * nside))
    c = oracle.radec2vec([200.0], [-40.0])[0]
    pix = np.nonzero(v @ c >= np.cos(np.radians(6.0)))[0]
    pick = rng.choice(pix, size=4000)                       # repeats: several galaxies per pixel
    pv = v[pick]
    ra = np.degrees(np.arctan2(pv[:, 1], pv[:, 0])) % 360.0
    dec = np.degrees(np.arcsin(pv[:, 2]))
    e1, e2 = rng.normal(0, 0.26, pick.size), rng.normal(0, 0.26, pick.size)
    w = rng.uniform(0.5, 1.5, pick.size)
    # targets on the coarser grid: their centres are never bin-pixel centres
    t64 = oracle.pix2vec(64, np.arange(12 * 64 * 64))
    tg = t64[t64 @ c >= np.cos(np.radians(5.0))]
    th = 50.0 * ARCMIN
    b = oracle.bin_catalog(nside, ra, dec, e1, e2, w)
    bc = oracle.barycentres(nside, ra, dec, w, b)
    # the barycentre of points at a pixel's centre is that centre
    np.testing.assert_allclose(bc["vec"], v[bc["pix"]], rtol=0, atol=1e-14)
    px = oracle.map_pixels(tg, nside, b["G1"], b["G2"], b["W"], b["S2"], b["n"], 2, th)
    pb = oracle.map_barycentre(tg, nside, ra, dec, e1, e2, w, 2, th)
    np.testing.assert_array_equal(pb["N"], px["N"])
    for k in ("ME", "MB", "VAR", "SW"):
        np.testing.assert_allclose(pb[k], px[k], rtol=1e-9, atol=1e-12)


def test_barycentre_is_the_weighted_mean_direction():
    # two galaxies in one pixel: the barycentre lies on the great-circle arc
    # between them, dividing it in the ratio of the weights (tan relation)
    nside = 4
    p0 = 100
    r = oracle.pix2vec(nside, [p0])[0]
    east = np.array([-r[1], r[0], 0.0]) / np.hypot(r[0], r[1])
    pa = r + 0.02 * east
    pb_ = r - 0.02 * east
    pts = np.stack([pa, pb_]) / np.linalg.norm(np.stack([pa, pb_]), axis=1)[:, None]
    ra = np.degrees(np.arctan2(pts[:, 1], pts[:, 0])) % 360.0
    dec = np.degrees(np.arcsin(pts[:, 2]))
    assert (oracle.ang2pix(nside, ra, dec) == p0).all()
    w = np.array([3.0, 1.0])
    b = oracle.bin_catalog(nside, ra, dec, np.zeros(2), np.zeros(2), w)
    bc = oracle.barycentres(nside, ra, dec, w, b)
    want = (3.0 * pts[0] + pts[1]) / np.linalg.norm(3.0 * pts[0] + pts[1])
    np.testing.assert_allclose(bc["vec"][0], want, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# averaged normalisation (Sect. 2.4)
# --------------------------------------------------------------------------
def test_averaged_equals_summed_times_pixel_area_ratio_for_equal_weights():
    # when every bin pixel carries the same weight W0, the averaged map is the
    # summed map times (members x pixel area) / aperture area, exactly
    nside = 64
    npix = 12 * nside * nside
    rng = np.random.default_rng(21)
    G1, G2 = rng.normal(0, 1, npix), rng.normal(0, 1, npix)
    W = np.full(npix, 7.0)
    S2 = rng.uniform(1, 2, npix)
    n_p = np.full(npix, 7, np.int64)
    tg = oracle.pix2vec(32, np.arange(0, 12 * 32 * 32, 97))
    th = 3.0 * np.pi / 180
    s = oracle.map_pixels(tg, nside, G1, G2, W, S2, n_p, 2, th)
    a = oracle.map_pixels_averaged(tg, nside, G1, G2, W, S2, n_p, 2, th)
    apix = 4 * np.pi / npix
    area = 2 * np.pi * (1 - np.cos(th))
    ratio = s["NPIX"] * apix / area
    np.testing.assert_allclose(a["ME"], s["ME"] * ratio, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(a["MB"], s["MB"] * ratio, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(a["VAR"], s["VAR"] * ratio ** 2, rtol=1e-12, atol=1e-18)


def test_averaged_map_of_a_smooth_field_approaches_the_integral():
    # averaged = the pixel discretisation of int gamma_+ Q dA: for a noiseless
    # isolated SIS the polynomial-filter map tends to the closed form of the
    # flat limit, 4 theta_E / (5 theta_ap), as pixels shrink
    nside = 1024
    te = 0.5 * ARCMIN
    th = 30.0 * ARCMIN
    ra0, dec0 = 0.0, 0.0
    tgt = oracle.radec2vec([ra0], [dec0])
    pix = oracle.query_disc(nside, tgt[0], th)
    v = oracle.pix2vec(nside, pix)
    # gamma_t = theta_E / (2 theta), tangential about the halo at the target
    x, y, z = v[:, 0], v[:, 1], v[:, 2]
    ra = np.arctan2(y, x)
    dec = np.arcsin(z)
    theta = 2 * np.arcsin(np.linalg.norm(v - tgt[0], axis=1) / 2)
    gt = np.where(theta > te, te / (2 * np.maximum(theta, 1e-300)), 0.5)
    # bearing of the halo (at ra0, dec0) from each pixel, from North through East
    b = np.arctan2(np.sin(-ra) * np.cos(0.0), np.cos(dec) * np.sin(0.0) - np.sin(dec) * np.cos(0.0) * np.cos(-ra))
    g1 = np.zeros(12 * nside * nside)
    g2 = np.zeros(12 * nside * nside)
    g1[pix] = gt * np.cos(2 * b)
    g2[pix] = -gt * np.sin(2 * b)
    W = np.ones(12 * nside * nside)
    a = oracle.map_pixels_averaged(tgt, nside, g1, g2, W, np.zeros_like(W), np.ones(W.size, np.int64), 1, th)
    assert abs(a["ME"][0] - 4 * te / (5 * th)) < 0.02 * 4 * te / (5 * th)
    assert abs(a["MB"][0]) < 1e-3 * 4 * te / (5 * th)


# --------------------------------------------------------------------------
# Jarvis et al. (2004) filter
# --------------------------------------------------------------------------
def _u_jarvis(x, s):
    """The compensated U of the Gaussian-type filter (theta_ap = 1, scale s)."""
    return (1.0 - x * x / (2 * s * s)) * np.exp(-x * x / (2 * s * s)) / (2 * np.pi * s * s)


def test_jarvis_q_follows_from_its_compensated_u():
    from scipy.integrate import quad
    s = 0.25
    # U is compensated over the whole plane: int_0^inf x U dx = 0
    comp, _ = quad(lambda t: t * _u_jarvis(t, s), 0, 40 * s, limit=200)
    assert abs(comp) < 1e-12
    # Eq. 5: Q = (2 / x^2) int_0^x x' U dx' - U
    for x in (0.05, 0.1, 0.25, 0.4, 0.7, 1.0):
        inner, _ = quad(lambda t: t * _u_jarvis(t, s), 0, x, epsabs=1e-14, epsrel=1e-12)
        q_from_u = 2.0 / (x * x) * inner - _u_jarvis(x, s)
        assert abs(oracle.filter_q(3, x, s) - q_from_u) < 1e-10 * max(1.0, abs(q_from_u))


# ------------------------------------------- noise map normalisation (Eq. 8)
def _noise_field(seed, theta_ap, per_target=600):
    """Fixed positions and weights around centres whose apertures do not
    overlap: pixel centres of an NSIDE 4 grid (spacing about 15 degrees) plus
    one aperture around each pole, so that polar geometry is in the sample."""
    rng = np.random.default_rng(seed)
    cen = oracle.pix2vec(4, np.arange(0, 192, 4))
    cen = np.concatenate([cen, oracle.radec2vec([17.0, 250.0], [89.93, -89.9])])
    ra, dec = [], []
    for c in cen:
        # uniform in a cap of radius 1.05 theta_ap about c
        cr = 1.0 - rng.random(per_target) * (1.0 - math.cos(1.05 * theta_ap))
        sr = np.sqrt(1.0 - cr * cr)
        ph = 2 * math.pi * rng.random(per_target)
        a = np.array([0.0, 0.0, 1.0]) if abs(c[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
        e_1 = np.cross(a, c)
        e_1 /= np.linalg.norm(e_1)
        e_2 = np.cross(c, e_1)
        v = cr[:, None] * c + sr[:, None] * (np.cos(ph)[:, None] * e_1 + np.sin(ph)[:, None] * e_2)
        ra.append(np.degrees(np.arctan2(v[:, 1], v[:, 0])) % 360)
        dec.append(np.degrees(np.arcsin(np.clip(v[:, 2], -1, 1))))
    ra, dec = np.concatenate(ra), np.concatenate(dec)
    w = rng.uniform(0.5, 1.5, ra.size)
    return cen, ra, dec, w, rng


@pytest.mark.parametrize("mode", ["galaxies", "pixels"])
def test_noise_map_normalisation_monte_carlo(mode):
    """Eq. 8 with weights: the noise map is the variance of M_E and M_B under
    pure shape noise.  With e1, e2 ~ N(0, s^2) independent, E|e|^2 = 2 s^2,
    so for fixed positions and weights Var(M_E) = Var(M_B) = (A / sum w)^2
    sum w^2 Q^2 s^2, which is the expectation of sigma^2 = SV / (2 nbar^2).
    The test draws many noise realisations through the oracle and compares
    the pooled sample second moment of M_E and M_B (mean zero) with the
    pooled mean of the oracle's sigma^2; a wrong factor 1/2, a w in place of
    w^2, or nbar in place of nbar^2 moves the ratio far from 1.  M_E and M_B
    are independent here (zero covariance, jointly Gaussian), so about
    2 x 50 x 400 samples fix the ratio to about 0.7 % (one sd).  Pixel mode
    bins each realisation (Sect. 3.2 step 2), so its S2 = sum w^2 |e|^2
    holds noise of the same expectation."""
    th = 20 * ARCMIN
    cen, ra, dec, w, rng = _noise_field(11, th)
    s = synth.SIGMA_E
    m2, var = 0.0, 0.0
    nreal = 400
    for _ in range(nreal):
        e1 = rng.normal(0.0, s, ra.size)
        e2 = rng.normal(0.0, s, ra.size)
        if mode == "galaxies":
            r = oracle.map_galaxies(cen, ra, dec, e1, e2, w, 1, th)
        else:
            b = oracle.bin_catalog(256, ra, dec, e1, e2, w)
            r = oracle.map_pixels(cen, 256, b["G1"], b["G2"], b["W"], b["S2"], b["n"], 1, th)
        assert np.all(r["N"] > 100)
        m2 += np.sum(r["ME"] ** 2 + r["MB"] ** 2)
        var += 2.0 * np.sum(r["VAR"])
    ratio = m2 / var
    assert abs(ratio - 1.0) < 0.04, ratio
