"""Seeded test inputs shared by the parity tests (built with the synth module)."""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle
from paper_2609_11181_b300 import synth

ARCMIN = math.pi / 10800.0


def cap_targets(nside: int, ra0: float, dec0: float, radius_deg: float) -> np.ndarray:
    """RING pixels at nside whose centres lie in the cap (oracle geometry)."""
    v = oracle.pix2vec(nside, np.arange(12 * nside * nside))
    c = oracle.radec2vec([ra0], [dec0])[0]
    return np.nonzero(v @ c >= math.cos(math.radians(radius_deg)))[0].astype(np.int64)


def catalog(seed: int, n: int, ra0: float, dec0: float, radius_deg: float, nhalo: int = 5,
            te=(0.2, 1.0), w_range=None, clumped=False, r_trunc_deg=2.0):
    g = synth.make_gen(seed)
    rad = math.radians(radius_deg)
    halos = synth.halos_uniform(nhalo, ra0, dec0, rad, g, te[0] * ARCMIN, te[1] * ARCMIN)
    cat = synth.galaxy_catalog(n, ra0, dec0, rad, halos, g, r_trunc=math.radians(r_trunc_deg),
                               w_range=w_range, clumped=clumped)
    return cat


def c1_catalog(n: int = 200_000, seed: int = 101):
    """Config: 10 deg cap at (0,0), uniform galaxies, 5 SIS (theta_E 0.2-1'), w = 1."""
    return catalog(seed, n, 0.0, 0.0, 10.0, nhalo=5)


def binned_from_catalog(nside: int, cat) -> dict:
    b = oracle.bin_catalog(nside, cat.ra_deg.numpy(), cat.dec_deg.numpy(), cat.e1.double().numpy(),
                           cat.e2.double().numpy(), cat.w.double().numpy())
    return b


def to_cuda(cat, dev):
    return cat.to(dev)


def binned_field_oracle(seed: int, nside: int, ra0: float, dec0: float, radius_deg: float,
                        mean_count: float, halo_density: float = 1.333, r_trunc_deg: float = 1.0):
    """Per-pixel binned shear (pixel-based workloads) at oracle pixel centres."""
    npix = 12 * nside * nside
    g = synth.make_gen(seed)
    rad = math.radians(radius_deg)
    area = 2 * math.pi * (1 - math.cos(rad)) * (180 / math.pi) ** 2
    halos = synth.halos_poisson(halo_density, area, ra0, dec0, rad, g)
    v = torch.from_numpy(oracle.pix2vec(nside, np.arange(npix)))
    c = torch.from_numpy(oracle.radec2vec([ra0], [dec0])[0])
    foot = (v @ c) >= math.cos(rad)
    b = synth.binned_field(v, foot, mean_count, halos, g, r_trunc=math.radians(r_trunc_deg))
    return b, foot.numpy()


def rms_rel(a, b):
    return oracle.rms_rel(np.asarray(a, np.float64), np.asarray(b, np.float64))
