"""GPU parity of the barycentre form of the pixel-based map (Sect. 3.3)
against the float64 oracle: member pixels and galaxy counts bit-exact, maps
within 1e-4 relative rms."""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_11181_b300 import api, synth

from _cases import ARCMIN, catalog, cap_targets, rms_rel

pytestmark = pytest.mark.gpu


def _check(got, ref, label):
    np.testing.assert_array_equal(got["count"].cpu().numpy(), ref["N"], err_msg=label + " counts")
    np.testing.assert_array_equal(got["members"].cpu().numpy(), ref["K"], err_msg=label + " members")
    np.testing.assert_allclose(got["sum_w"].cpu().numpy(), ref["SW"], rtol=1e-6, atol=1e-12)
    for k_got, k_ref in (("map_e", "ME"), ("map_b", "MB"), ("var", "VAR")):
        e = rms_rel(got[k_got].cpu().numpy(), ref[k_ref])
        assert e <= 1e-4, f"{label} {k_got}: {e:.3e}"


@pytest.mark.parametrize("ra0,dec0,rad,no,nb,th,filt", [
    (40.0, 10.0, 3.0, 256, 512, 20.0, "schirmer"),
    (355.0, 60.0, 3.0, 128, 256, 30.0, "poly"),       # RA wrap, polar rings
    (200.0, -89.0, 2.0, 256, 256, 15.0, "schirmer"),  # south pole
])
def test_barycentre_map_matches_oracle(cuda_device, ra0, dec0, rad, no, nb, th, filt):
    kind = 1 if filt == "poly" else 2
    cat = catalog(int(ra0 + 7 * dec0 + 500), 80_000, ra0, dec0, rad + th / 60.0, nhalo=5, w_range=(0.5, 1.5),
                  clumped=True)
    tg = cap_targets(no, ra0, dec0, rad)
    ctx = api.Context(no, th, filt, nside_bin=nb)
    ctx.set_targets(torch.from_numpy(tg).to(cuda_device))
    c = cat.to(cuda_device)
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    got = ctx.map_barycentre()
    ctx.sync(60)
    ref = oracle.map_barycentre(oracle.pix2vec(no, tg), nb, cat.ra_deg.numpy(), cat.dec_deg.numpy(),
                                cat.e1.double().numpy(), cat.e2.double().numpy(), cat.w.double().numpy(), kind,
                                th * ARCMIN)
    _check(got, ref, "barycentre")


def test_barycentre_records_follow_the_catalogue(cuda_device):
    # a second catalogue on the same context rebuilds the records
    tg = cap_targets(128, 100.0, 30.0, 2.0)
    ctx = api.Context(128, 25.0, "poly", nside_bin=256)
    ctx.set_targets(torch.from_numpy(tg).to(cuda_device))
    for seed in (61, 62):
        cat = catalog(seed, 30_000, 100.0, 30.0, 2.6, nhalo=3)
        c = cat.to(cuda_device)
        ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
        got = ctx.map_barycentre()
        ctx.sync(60)
        ref = oracle.map_barycentre(oracle.pix2vec(128, tg), 256, cat.ra_deg.numpy(), cat.dec_deg.numpy(),
                                    cat.e1.double().numpy(), cat.e2.double().numpy(), cat.w.double().numpy(), 1,
                                    25.0 * ARCMIN)
        _check(got, ref, f"catalogue {seed}")


def test_barycentre_map_equals_brute_force_with_sparse_catalogue(cuda_device):
    # at most one galaxy per bin pixel: every barycentre is its galaxy
    full = catalog(63, 3_000, 250.0, -20.0, 2.0)
    pix = oracle.ang2pix(8192, full.ra_deg.numpy(), full.dec_deg.numpy())
    _, first = np.unique(pix, return_index=True)          # one galaxy per pixel
    keep = torch.from_numpy(np.sort(first))
    cat = synth.Catalog(*(getattr(full, k)[keep] for k in ("ra_deg", "dec_deg", "e1", "e2", "w")))
    tg = cap_targets(256, 250.0, -20.0, 1.5)
    ctx = api.Context(256, 20.0, "schirmer", nside_bin=8192)
    ctx.set_targets(torch.from_numpy(tg).to(cuda_device))
    c = cat.to(cuda_device)
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    bf = ctx.map_bruteforce()
    bf = {k: v.clone() for k, v in bf.items()}
    pb = ctx.map_barycentre()
    ctx.sync(60)
    assert torch.equal(bf["count"], pb["count"]) and torch.equal(bf["count"].int(), pb["members"])
    for k in ("map_e", "map_b", "var"):
        assert rms_rel(pb[k].cpu().numpy(), bf[k].cpu().numpy()) <= 1e-5, k
