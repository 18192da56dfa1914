"""GPU parity of catalogue partitioning (Sect. 3.4) and binning (Sect. 3.2
step 2): pixel of every galaxy, the stable sort permutation, the offset table
and the per-pixel counts bit-exact; per-pixel float32 sums within float32
rounding of the float64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2609_11181_b300 import api
from paper_2609_11181_b300._native import SmartError

from _cases import boundary_points, catalog

pytestmark = pytest.mark.gpu


def _run(cuda_device, cat, nside, only_counts=False):
    ctx = api.Context(nside, 10.0, "poly", nside_bin=nside)
    c = cat.to(cuda_device)
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    perm, pix, off = ctx.get_catalog(cat.n)
    b = ctx.get_binned()
    if only_counts:
        b = {"n": b["n"]}
    ctx.sync(60)
    return ctx, perm.cpu().numpy(), pix.cpu().numpy(), off.cpu().numpy(), {k: v.cpu().numpy() for k, v in b.items()}


@pytest.mark.parametrize("n,nside,clumped", [(1, 16, False), (4095, 64, False), (4096 * 3 + 123, 256, True),
                                             (300_000, 1024, True)])
def test_sort_and_bins_match_oracle(cuda_device, n, nside, clumped):
    cat = catalog(n + nside, n, 33.0, -12.0, 6.0, nhalo=8, w_range=(0.5, 1.5), clumped=clumped)
    ctx, perm, pix, off, b = _run(cuda_device, cat, nside)
    ref = oracle.bin_catalog(nside, cat.ra_deg.numpy(), cat.dec_deg.numpy(), cat.e1.double().numpy(),
                             cat.e2.double().numpy(), cat.w.double().numpy())
    np.testing.assert_array_equal(perm, ref["perm"])
    np.testing.assert_array_equal(pix, ref["pix"][ref["perm"]])
    np.testing.assert_array_equal(off, ref["offsets"])
    np.testing.assert_array_equal(b["n"], ref["n"])
    # float32 sums of float32 terms in the same order: error <= n_p * 2^-23 * sum |term|
    w = cat.w.double().numpy()
    absG = np.bincount(ref["pix"], w * np.abs(cat.e1.double().numpy()), len(ref["n"]))
    tol = (ref["n"] + 1) * 1.2e-7 * absG + 1e-30
    assert np.all(np.abs(b["G1"] - ref["G1"]) <= tol)
    np.testing.assert_allclose(b["W"], ref["W"], rtol=(ref["n"].max() + 1) * 1.2e-7)
    np.testing.assert_allclose(b["S2"], ref["S2"], rtol=(ref["n"].max() + 1) * 1.2e-7 + 1e-6)
    ctx.close()


def test_sort_large_nside(cuda_device):
    # nside 4096 (28-bit keys, four radix passes): permutation and offsets
    n = 1_500_000
    cat = catalog(77, n, 250.0, 55.0, 8.0, nhalo=8, w_range=(0.5, 1.5), clumped=True)
    nside = 4096
    ctx, perm, pix, off, b = _run(cuda_device, cat, nside, only_counts=True)
    ref_pix = oracle.ang2pix(nside, cat.ra_deg.numpy(), cat.dec_deg.numpy())
    ref_perm = np.argsort(ref_pix, kind="stable")
    np.testing.assert_array_equal(perm, ref_perm)
    sp = ref_pix[ref_perm]
    np.testing.assert_array_equal(pix, sp)
    rng = np.random.default_rng(0)
    probe = np.unique(np.concatenate([sp[rng.integers(0, n, 5000)], rng.integers(0, 12 * nside ** 2, 5000),
                                      [0, 12 * nside ** 2]]))
    np.testing.assert_array_equal(off[probe], np.searchsorted(sp, probe, side="left"))
    cnt = np.bincount(ref_pix, minlength=12 * nside ** 2)
    np.testing.assert_array_equal(b["n"], cnt)
    ctx.close()


def test_sort_is_stable_for_identical_positions(cuda_device):
    # many galaxies at exactly the same place: the permutation keeps input order
    n = 20000
    ra = np.full(n, 12.5)
    dec = np.full(n, -3.25)
    ra[::3] = 200.0
    e = np.zeros(n, np.float32)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(cuda_device, dt)
    ctx = api.Context(64, 10.0, nside_bin=4096)
    ctx.bin_galaxies(t(ra, torch.float64), t(dec, torch.float64), t(e, torch.float32), t(e, torch.float32), None)
    perm, pix, off = ctx.get_catalog(n)
    ctx.sync(60)
    pix_ref = oracle.ang2pix(4096, ra, dec)
    np.testing.assert_array_equal(perm.cpu().numpy(), np.argsort(pix_ref, kind="stable"))


def test_empty_catalog(cuda_device):
    ctx = api.Context(16, 30.0, nside_bin=16)
    e64 = torch.empty(0, dtype=torch.float64, device=cuda_device)
    e32 = torch.empty(0, dtype=torch.float32, device=cuda_device)
    ctx.bin_galaxies(e64, e64, e32, e32, e32)
    b = ctx.get_binned()
    _, _, off = ctx.get_catalog(0)
    ctx.sync(60)
    assert int(b["n"].sum()) == 0 and int(off.abs().sum()) == 0


def test_invalid_coordinates_rejected(cuda_device):
    # the call does not wait; the device counts the two invalid galaxies, the
    # next sync reports them (SMART_E_ARG), and they are left out of the
    # catalogue; the sync after that is clean
    ctx = api.Context(16, 30.0, nside_bin=16)
    ra = torch.tensor([10.0, float("nan"), 20.0], dtype=torch.float64, device=cuda_device)
    dec = torch.tensor([0.0, 0.0, 95.0], dtype=torch.float64, device=cuda_device)
    e = torch.zeros(3, dtype=torch.float32, device=cuda_device)
    ctx.bin_galaxies(ra, dec, e, e, None)
    with pytest.raises(SmartError, match="2 galaxies") as err:
        ctx.sync(60)
    assert "SMART_E_ARG" in str(err.value)
    perm, pix, off = ctx.get_catalog(3)
    ctx.sync(60)
    assert int(off[-1]) == 1 and int(perm[0]) == 0


@pytest.mark.parametrize("nside", [1, 16, 256, 4096, 8192])
def test_keys_at_pixel_boundaries(cuda_device, nside):
    # the catalogue's pixel keys come from float32 trigonometry where that
    # decision is certain and from the float64 definition elsewhere: on points
    # placed at every kind of pixel boundary they still equal the oracle
    ra, dec = boundary_points(nside, 40_000, nside)
    n = ra.size
    ctx = api.Context(nside, 10.0, "poly", nside_bin=nside)
    t = lambda x, dt: torch.from_numpy(np.ascontiguousarray(x)).to(cuda_device, dt)
    ones = torch.ones(n, dtype=torch.float32, device=cuda_device)
    ctx.bin_galaxies(t(ra, torch.float64), t(dec, torch.float64), ones, ones, ones)
    perm, pix, off = ctx.get_catalog(n)
    ctx.sync(60)
    ref = oracle.ang2pix(nside, ra, dec)
    ref_perm = np.argsort(ref, kind="stable")
    np.testing.assert_array_equal(pix.cpu().numpy(), ref[ref_perm])
    np.testing.assert_array_equal(perm.cpu().numpy(), ref_perm)
    ctx.close()
