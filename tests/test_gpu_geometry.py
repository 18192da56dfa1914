"""GPU parity of the device HEALPix geometry: pixel indices and pixel-centre
unit vectors must be bit-identical to the float64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_11181_b300 import api

pytestmark = pytest.mark.gpu


def _points(n, seed):
    rng = np.random.default_rng(seed)
    ra = rng.uniform(-720, 720, n)
    dec = np.degrees(np.arcsin(rng.uniform(-1, 1, n)))
    edge_ra = np.array([0.0, 90.0, 180.0, 270.0, 360.0, -0.0, 45.0, 1e-300, 359.99999999999994])
    edge_dec = np.array([90.0, -90.0, 0.0, 41.810314895778596, -41.810314895778596, 89.9999999, -89.9999999,
                         1e-300, 30.0])
    ra = np.concatenate([ra, edge_ra, np.repeat(edge_ra, len(edge_dec))])
    dec = np.concatenate([dec, edge_dec, np.tile(edge_dec, len(edge_ra))])
    return ra, dec


@pytest.mark.parametrize("nside", [1, 2, 16, 256, 2048, 4096, 8192])
def test_ang2pix_bit_exact(cuda_device, nside):
    ra, dec = _points(200_000, nside)
    got = api.ang2pix(nside, torch.from_numpy(ra).to(cuda_device), torch.from_numpy(dec).to(cuda_device))
    ref = oracle.ang2pix(nside, ra, dec)
    np.testing.assert_array_equal(got.cpu().numpy(), ref)


@pytest.mark.parametrize("nside", [1, 4, 64, 1024, 4096, 8192])
def test_pix2vec_bit_exact(cuda_device, nside):
    npix = 12 * nside * nside
    rng = np.random.default_rng(nside)
    pix = np.unique(np.concatenate([rng.integers(0, npix, 100_000), np.arange(min(npix, 5000)),
                                    np.arange(max(0, npix - 5000), npix),
                                    np.arange(2 * nside * (nside - 1) - 10, 2 * nside * (nside - 1) + 10) % npix]))
    got = api.pix2vec(nside, torch.from_numpy(pix).to(cuda_device)).cpu().numpy()
    ref = oracle.pix2vec(nside, pix)
    np.testing.assert_array_equal(got, ref)


def test_pix2vec_out_of_range_is_nan(cuda_device):
    pix = torch.tensor([-1, 12 * 16 * 16, 5], dtype=torch.int64, device=cuda_device)
    v = api.pix2vec(16, pix).cpu().numpy()
    assert np.isnan(v[0]).all() and np.isnan(v[1]).all() and np.isfinite(v[2]).all()


def test_empty_inputs(cuda_device):
    e = torch.empty(0, dtype=torch.float64, device=cuda_device)
    assert api.ang2pix(64, e, e).numel() == 0
    assert api.pix2vec(64, torch.empty(0, dtype=torch.int64, device=cuda_device)).shape == (0, 3)
