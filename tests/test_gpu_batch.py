"""Batched pixel-based maps (one persistent launch in a CUDA graph) against
the single-map launches and the float64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2609_11181_b300 import api
from paper_2609_11181_b300._native import SmartError

from _cases import ARCMIN, binned_field_oracle, rms_rel

pytestmark = pytest.mark.gpu


def _problems(dev, specs):
    ctxs, data = [], []
    for seed, nside, ra0, dec0, rad, th, filt in specs:
        b, foot = binned_field_oracle(seed, nside, ra0, dec0, rad, mean_count=20.0)
        tg = torch.from_numpy(np.nonzero(foot)[0].astype(np.int64)).to(dev)
        px = torch.stack([b.G1, b.G2, b.S2, b.W], dim=1).contiguous().to(dev)
        n = b.n.to(dev)
        ctx = api.Context(nside, th, filt, nside_bin=nside)
        ctx.set_targets(tg)
        ctx.set_binned_packed(px, n)
        ctxs.append(ctx)
        data.append((b, foot, px, n, th, nside))
    return ctxs, data


SPECS = [
    (11, 128, 20.0, 10.0, 12.0, 40.0, "schirmer"),     # equatorial: Toeplitz tiles
    (12, 128, 100.0, 70.0, 10.0, 60.0, "schirmer"),    # polar: general targets
    (13, 256, 250.0, -35.0, 6.0, 20.0, "schirmer"),
    (14, 64, 300.0, 85.0, 8.0, 90.0, "schirmer"),      # around the pole
]


def test_batch_equals_single_maps(cuda_device):
    ctxs, data = _problems(cuda_device, SPECS)
    singles = [c.map_pixel() for c in ctxs]
    torch.cuda.synchronize()
    # the polar caps have general targets in mirror pairs
    assert all(ctxs[i].general_pairs()[0].shape[0] > 0 for i in (1, 3))
    batch = api.Batch(ctxs, autotune=True)
    outs = batch.run()
    torch.cuda.synchronize()
    info = batch.info()
    assert info["n_items"] > 0 and info["ctas_per_sm"] in (7, 8, 9, 10, 11, 12)
    for s, o in zip(singles, outs):
        for k in ("map_e", "map_b", "var", "sum_w", "count", "members"):
            assert torch.equal(s[k], o[k]), k
    # replaying the graph gives the same maps
    before = [o["map_e"].clone() for o in outs]
    batch.run()
    torch.cuda.synchronize()
    for x, o in zip(before, outs):
        assert torch.equal(x, o["map_e"])
    batch.close()


def test_batch_against_oracle_and_borrowed_inputs(cuda_device):
    ctxs, data = _problems(cuda_device, SPECS[:2])
    batch = api.Batch(ctxs, autotune=False)
    outs = batch.run()
    torch.cuda.synchronize()
    for o, (b, foot, px, n, th, nside) in zip(outs, data):
        tg = np.nonzero(foot)[0]
        ref = oracle.map_pixels(oracle.pix2vec(nside, tg), nside, b.G1.double().numpy(), b.G2.double().numpy(),
                                b.W.double().numpy(), b.S2.double().numpy(), b.n.long().numpy(), 2, th * ARCMIN)
        np.testing.assert_array_equal(o["count"].cpu().numpy(), ref["N"])
        assert rms_rel(o["map_e"].cpu().numpy(), ref["ME"]) <= 1e-4
    # the graph reads the borrowed packed map at run time: flip the shear
    for (_, _, px, _, _, _) in data:
        px[:, 0:2].neg_()
    e0 = [o["map_e"].clone() for o in outs]
    batch.run()
    torch.cuda.synchronize()
    for x, o in zip(e0, outs):
        assert torch.allclose(o["map_e"], -x, rtol=1e-6, atol=1e-6 * float(x.abs().max()))
    batch.close()


def test_batch_rejects_mixed_filters(cuda_device):
    specs = [SPECS[0], (15, 64, 0.0, 0.0, 5.0, 30.0, "poly")]
    ctxs, _ = _problems(cuda_device, specs)
    with pytest.raises(SmartError):
        api.Batch(ctxs)
