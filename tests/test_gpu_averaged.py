"""GPU parity of the averaged normalisation (Sect. 2.4) against the float64
oracle, for the pixel-based, barycentre and brute-force maps: counts
bit-exact, maps within 1e-4 relative rms."""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_11181_b300 import api

from _cases import ARCMIN, binned_field_oracle, catalog, cap_targets, rms_rel

pytestmark = pytest.mark.gpu


def _check(got, ref, label):
    np.testing.assert_array_equal(got["count"].cpu().numpy(), ref["N"], err_msg=label + " counts")
    for k_got, k_ref in (("map_e", "ME"), ("map_b", "MB"), ("var", "VAR")):
        e = rms_rel(got[k_got].cpu().numpy(), ref[k_ref])
        assert e <= 1e-4, f"{label} {k_got}: {e:.3e}"


def test_averaged_pixel_map(cuda_device):
    nside = 256
    b, foot = binned_field_oracle(41, nside, 60.0, 50.0, 5.0, mean_count=8.0)
    tg = np.nonzero(foot)[0].astype(np.int64)
    ctx = api.Context(nside, 25.0, "schirmer", nside_bin=nside)
    ctx.set_targets(torch.from_numpy(tg).to(cuda_device))
    ctx.set_binned(*(x.to(cuda_device) for x in (b.G1, b.G2, b.W, b.S2, b.n)))
    ctx.set_normalisation("averaged")
    got = ctx.map_pixel()
    ctx.sync(60)
    ref = oracle.map_pixels_averaged(oracle.pix2vec(nside, tg), nside, b.G1.double().numpy(), b.G2.double().numpy(),
                                     b.W.double().numpy(), b.S2.double().numpy(), b.n.long().numpy(), 2,
                                     25.0 * ARCMIN)
    _check(got, ref, "pixel")
    # back to the summed form on the same context
    ctx.set_normalisation("summed")
    got2 = ctx.map_pixel()
    ctx.sync(60)
    ref2 = oracle.map_pixels(oracle.pix2vec(nside, tg), nside, b.G1.double().numpy(), b.G2.double().numpy(),
                             b.W.double().numpy(), b.S2.double().numpy(), b.n.long().numpy(), 2, 25.0 * ARCMIN)
    _check(got2, ref2, "pixel summed")


@pytest.mark.parametrize("mode", ["brute", "barycentre"])
def test_averaged_catalogue_maps(cuda_device, mode):
    cat = catalog(42, 60_000, 310.0, -25.0, 3.3, nhalo=4, w_range=(0.5, 1.5), clumped=True)
    tg = cap_targets(256, 310.0, -25.0, 2.8)
    ctx = api.Context(256, 20.0, "poly", nside_bin=512)
    ctx.set_targets(torch.from_numpy(tg).to(cuda_device))
    c = cat.to(cuda_device)
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    ctx.set_normalisation("averaged")
    got = ctx.map_bruteforce() if mode == "brute" else ctx.map_barycentre()
    ctx.sync(60)
    args = (oracle.pix2vec(256, tg), 512, cat.ra_deg.numpy(), cat.dec_deg.numpy(), cat.e1.double().numpy(),
            cat.e2.double().numpy(), cat.w.double().numpy(), 1, 20.0 * ARCMIN)
    ref = oracle.map_galaxies_averaged(*args) if mode == "brute" else oracle.map_barycentre_averaged(*args)
    _check(got, ref, mode)


def test_batch_rejects_averaged_contexts(cuda_device):
    nside = 64
    b, foot = binned_field_oracle(43, nside, 0.0, 0.0, 10.0, mean_count=5.0)
    ctx = api.Context(nside, 60.0, "schirmer", nside_bin=nside)
    ctx.set_targets(torch.from_numpy(np.nonzero(foot)[0].astype(np.int64)).to(cuda_device))
    ctx.set_binned(*(x.to(cuda_device) for x in (b.G1, b.G2, b.W, b.S2, b.n)))
    ctx.set_normalisation("averaged")
    with pytest.raises(api.SmartError):
        api.Batch([ctx], autotune=False)
