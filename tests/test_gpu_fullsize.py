"""Parity at the benchmark's full sizes, in the benchmark's launch
configuration, on targets sampled from the full maps.

The whole map is computed on the GPU exactly as bench.py does (packed
binned input for the NSIDE 4096 pixel map; catalogue sort + brute force
for the 5e7-galaxy map); the float64 oracle then computes a seeded random
sample of the targets one by one on the host.  Inputs are generated with the
oracle's pixel centres, so no oracle input comes from the CUDA path.

Bars as elsewhere: counts bit-exact; rms(M_gpu - M_oracle) / rms(M_oracle)
<= 1e-4 over the sample for M_E, M_B and sigma^2; weight sums within 1e-6.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2609_11181_b300 import api, workloads

from _cases import ARCMIN, rms_rel

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _oracle_centres(nside, p):
    return torch.from_numpy(oracle.pix2vec(nside, p.cpu().numpy())).to(p.device)


def _compare(got, ref, idx):
    np.testing.assert_array_equal(got["count"][idx], ref["N"])
    np.testing.assert_allclose(got["sum_w"][idx], ref["SW"], rtol=1e-6, atol=1e-12)
    for k_got, k_ref in (("map_e", "ME"), ("map_b", "MB"), ("var", "VAR")):
        e = rms_rel(got[k_got][idx].astype(np.float64), ref[k_ref])
        assert e <= TOL, f"{k_got}: rms rel err {e:.3e}"


def test_pixel4096_full_map_sampled(cuda_device):
    """15,000 deg^2 at NSIDE 4096, Schirmer 10': all 7.3e7 targets on the GPU,
    2,000 sampled targets (both pixel kernels) checked against the oracle."""
    wl = workloads.pixel_workload(cuda_device, _oracle_centres, **workloads.PIXEL_WORKLOADS["pixel4096"])
    host = [x.cpu().numpy() for x in (wl.G1, wl.G2, wl.W, wl.S2, wl.n)]
    px = torch.stack([wl.G1, wl.G2, wl.S2, wl.W], dim=1).contiguous()
    n_p = wl.n
    del wl.G1, wl.G2, wl.S2, wl.W
    ctx = api.Context(wl.nside, wl.theta_ap_arcmin, wl.filter, nside_bin=wl.nside)
    ctx.set_targets(wl.targets)
    ctx.set_binned_packed(px, n_p)
    out = ctx.map_pixel()
    ctx.sync(300)
    gen = ctx.general_targets().cpu().numpy()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    tg = wl.targets.cpu().numpy()
    ctx.close()
    del px, out
    torch.cuda.empty_cache()
    rng = np.random.default_rng(4096)
    # half the sample from the general kernel's targets, half from the Toeplitz kernel's
    is_gen = np.zeros(tg.size, bool)
    is_gen[gen] = True
    idx = np.sort(np.concatenate([rng.choice(np.nonzero(is_gen)[0], 1000, replace=False),
                                  rng.choice(np.nonzero(~is_gen)[0], 1000, replace=False)]))
    cv = oracle.pix2vec(wl.nside, tg[idx])
    ref = oracle.finalise(oracle.aperture_pixels_f32(cv, wl.nside, *host, 2, wl.theta_ap_arcmin * ARCMIN),
                          wl.theta_ap_arcmin * ARCMIN)
    _compare(got, ref, idx)
    np.testing.assert_array_equal(got["members"][idx], ref["NPIX"])


def test_brute2048_full_map_sampled(cuda_device):
    """5e7 clustered galaxies on 1,000 deg^2, sorted into NSIDE 4096, output
    NSIDE 2048, polynomial 15': every target on the GPU, 400 sampled targets
    checked against the oracle's sum over the whole catalogue."""
    wl = workloads.galaxy_workload(cuda_device, _oracle_centres, **workloads.GALAXY_WORKLOADS["brute2048"])
    c = wl.cat
    ctx = api.Context(wl.nside_out, wl.theta_ap_arcmin, wl.filter, nside_bin=wl.nside_bin)
    ctx.set_targets(wl.targets)
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    out = ctx.map_bruteforce()
    ctx.sync(300)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    tg = wl.targets.cpu().numpy()
    ra, dec = c.ra_deg.cpu().numpy(), c.dec_deg.cpu().numpy()
    e1, e2, w = (x.double().cpu().numpy() for x in (c.e1, c.e2, c.w))
    ctx.close()
    del c, wl.cat
    torch.cuda.empty_cache()
    idx = np.sort(np.random.default_rng(2048).choice(tg.size, 400, replace=False))
    cv = oracle.pix2vec(wl.nside_out, tg[idx])
    ref = oracle.map_galaxies(cv, ra, dec, e1, e2, w, 1, wl.theta_ap_arcmin * ARCMIN)
    _compare(got, ref, idx)
