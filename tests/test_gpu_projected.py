"""GPU parity of the Cartesian (projected) estimator, projS_pos (Sect. 2.2,
Sect. 5.2.1), and of the equal-area annulus statistics (Sect. 5.2.2),
against the float64 oracle.

Bar as for the spherical maps: member counts bit-exact; rms(M_gpu -
M_oracle) / rms(M_oracle) <= 1e-4 for M_E, M_B and sigma^2; weight sums
within 1e-6.  The geometry cases cover a reference point at mid latitude,
a wide field reaching 20 degrees from it (plane coordinates up to 0.36,
where the float32 hi/lo split of the positions matters), a reference point
near a pole with the RA seam inside the field, targets that have no image
(more than 90 degrees away: zeros), and both filter kinds.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2609_11181_b300 import api

from _cases import ARCMIN, cap_targets, catalog, rms_rel

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _check(got, ref, label=""):
    np.testing.assert_array_equal(got["count"].cpu().numpy(), ref["N"], err_msg=label + " counts")
    np.testing.assert_array_equal(got["members"].cpu().numpy(), ref["N"], err_msg=label + " members")
    np.testing.assert_allclose(got["sum_w"].cpu().numpy(), ref["SW"], rtol=1e-6, atol=1e-12, err_msg=label + " sum_w")
    for k_got, k_ref in (("map_e", "ME"), ("map_b", "MB"), ("var", "VAR")):
        e = rms_rel(got[k_got].cpu().numpy(), ref[k_ref])
        assert e <= TOL, f"{label} {k_got}: rms rel err {e:.3e}"


def _run(dev, cat, targets, nside_out, nside_bin, theta_arcmin, filt, ra_c, dec_c):
    ctx = api.Context(nside_out, theta_arcmin, filt, nside_bin=nside_bin)
    c = cat.to(dev)
    ctx.set_targets(torch.from_numpy(targets).to(dev))
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    out = ctx.map_projected(ra_c, dec_c)
    ctx.sync(120)
    return ctx, out


def _oracle(cat, targets, nside_out, theta_arcmin, kind, ra_c, dec_c):
    cv = oracle.pix2vec(nside_out, targets)
    return oracle.map_projected(cv, cat.ra_deg.numpy(), cat.dec_deg.numpy(), cat.e1.double().numpy(),
                                cat.e2.double().numpy(), cat.w.double().numpy(), ra_c, dec_c, kind,
                                theta_arcmin * ARCMIN)


@pytest.mark.parametrize("ra0,dec0,rad,no,nb,th,filt", [
    (40.0, 35.0, 4.0, 256, 1024, 20.0, "poly"),          # mid latitude
    (40.0, 35.0, 4.0, 256, 512, 20.0, "schirmer"),
    (200.0, -10.0, 20.0, 64, 256, 40.0, "schirmer"),     # wide field: plane coordinates up to 0.36
    (5.0, 80.0, 6.0, 128, 512, 30.0, "poly"),            # near the pole, RA seam inside the field
])
def test_projected_map_matches_oracle(cuda_device, ra0, dec0, rad, no, nb, th, filt):
    kind = 1 if filt == "poly" else 2
    cat = catalog(int(ra0 * 5 + dec0 * 11 + 77), 120_000, ra0, dec0, rad + th / 60.0, nhalo=6,
                  w_range=(0.5, 1.5), clumped=True)
    tg = cap_targets(no, ra0, dec0, rad)
    ctx, got = _run(cuda_device, cat, tg, no, nb, th, filt, ra0, dec0)
    ref = _oracle(cat, tg, no, th, kind, ra0, dec0)
    _check(got, ref, f"({ra0},{dec0})")
    assert ref["N"].min() > 0
    ctx.close()


def test_targets_without_image_and_offset_reference(cuda_device):
    """A reference point 3 degrees from the field's centre, plus targets
    more than 90 degrees away (no image: all outputs zero)."""
    cat = catalog(91, 50_000, 120.0, 20.0, 3.5, nhalo=4, w_range=(0.5, 1.5))
    near = cap_targets(256, 120.0, 20.0, 3.0)
    far = cap_targets(256, 300.0, -20.0, 0.5)          # the antipode of the field
    tg = np.sort(np.concatenate([near, far]))
    ctx, got = _run(cuda_device, cat, tg, 256, 512, 15.0, "schirmer", 118.0, 22.0)
    ref = _oracle(cat, tg, 256, 15.0, 2, 118.0, 22.0)
    _check(got, ref, "offset reference")
    is_far = np.isin(tg, far)
    assert np.all(got["count"].cpu().numpy()[is_far] == 0)
    assert np.all(got["map_e"].cpu().numpy()[is_far] == 0)
    ctx.close()


def test_projected_near_the_reference_point_approaches_spherical(cuda_device):
    """Sect. 5.2.2: the projected and spherical maps agree near the
    projection centre and drift apart with distance from it."""
    ra0, dec0, th = 60.0, 30.0, 10.0
    cat = catalog(93, 400_000, ra0, dec0, 8.5, nhalo=20, w_range=(0.5, 1.5))
    tg = cap_targets(512, ra0, dec0, 8.0)
    ctx, proj = _run(cuda_device, cat, tg, 512, 1024, th, "poly", ra0, dec0)
    sph = ctx.map_bruteforce()
    st = ctx.annulus_stats(ra0, dec0, math.radians(8.0), proj["map_e"], sph["map_e"], 8)
    ctx.sync(120)
    sd = st["sd"].cpu().numpy()
    assert sd[0] < sd[-1]
    assert np.all(np.diff(sd[1:]) > 0)
    ctx.close()


def test_annulus_stats_match_oracle(cuda_device):
    """Annulus statistics of two given maps (random, not from the library)."""
    nside, ra0, dec0 = 256, 10.0, -40.0
    tg = cap_targets(nside, ra0, dec0, 12.0)
    rng = np.random.default_rng(17)
    mref = rng.normal(0.0, 2e-3, tg.size).astype(np.float32)
    d = oracle.pix2vec(nside, tg) @ oracle.radec2vec([ra0], [dec0])[0]
    mx = (mref + rng.normal(0.0, 1e-4, tg.size) * (1 - d) * 1e3).astype(np.float32)
    rmax, nb = math.radians(11.0), 12
    ref = oracle.annulus_stats(oracle.pix2vec(nside, tg), oracle.radec2vec([ra0], [dec0])[0], rmax,
                               mx.astype(np.float64), mref.astype(np.float64), nb)
    ctx = api.Context(nside, 10.0, "poly", nside_bin=nside)
    ctx.set_targets(torch.from_numpy(tg).to(cuda_device))
    got = ctx.annulus_stats(ra0, dec0, rmax, torch.from_numpy(mx).to(cuda_device),
                            torch.from_numpy(mref).to(cuda_device), nb)
    ctx.sync(60)
    np.testing.assert_array_equal(got["count"].cpu().numpy(), ref["count"])
    np.testing.assert_allclose(got["mean"].cpu().numpy(), ref["mean"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(got["sd"].cpu().numpy(), ref["sd"], rtol=1e-9, atol=1e-12)
    ctx.close()
