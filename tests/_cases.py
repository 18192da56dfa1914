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


def boundary_points(nside, n, seed):
    """Points on and next to the pixel boundaries of the RING scheme: every
    floor of the definition (equatorial N(1/2 + t) -+ 3/4 N z, polar
    t_p N sqrt(3(1 - |z|)) and (1 - t_p) N sqrt(3(1 - |z|)), the azimuth index
    t i) lands within 0 .. 1e-3 of an integer or just past the float32 path's
    margins (1.5e-6 N .. 1e-5 N), plus |z| = 2/3 and the 0/360 azimuth seam;
    dec in degrees, ra in [-360, 720)."""
    rng = np.random.default_rng(seed)
    N = float(nside)
    offs = np.array([0.0, 1e-13, -1e-13, 1e-9, -1e-9, 1e-7, -1e-7, 1e-5, -1e-5, 1e-3, -1e-3] +
                    [f * N for f in (1.5e-6, -1.5e-6, 4e-6, -4e-6, 7e-6, -7e-6, 1e-5, -1e-5)])   # around the float32 margins
    ra, z = [], []
    tt = rng.uniform(0.0, 4.0, n)
    d = rng.choice(offs, n)
    # equatorial: v1 = N (1/2 + t) - 3/4 N z = m + d  or  v2 = N (1/2 + t) + 3/4 N z = m + d
    m = np.round(N * (0.5 + tt) + rng.uniform(-0.5, 0.5, n) * 1.5 * N * 2 / 3)
    sgn = rng.choice([-1.0, 1.0], n)
    ze = sgn * (m + d - N * (0.5 + tt)) / (0.75 * N)
    ok = np.abs(ze) <= 2.0 / 3.0
    ra.append(tt[ok] * 90.0), z.append(ze[ok])
    # polar: t_p N sqrt(3 (1 - za)) = m + d  (or with 1 - t_p); sign of z random
    tp = rng.uniform(0.0, 1.0, n)
    q = np.floor(rng.uniform(0, 4, n))
    side = rng.choice([0, 1], n)
    f = np.where(side == 0, tp, 1.0 - tp)
    mm = np.maximum(1.0, np.round(rng.uniform(0, 1, n) * N * f))
    za = 1.0 - ((mm + d) / np.maximum(f * N, 1e-300)) ** 2 / 3.0
    ok = (za > 2.0 / 3.0) & (za <= 1.0) & (f > 1e-6)
    ra.append((q[ok] + tp[ok]) * 90.0), z.append(za[ok] * rng.choice([-1.0, 1.0], ok.sum()))
    # polar azimuth index: t i = m + d on ring i
    i = rng.integers(1, max(2, nside), n)
    za = 1.0 - (i / N) ** 2 / 3.0
    jj = rng.integers(0, 4 * i)
    ra.append(((jj + d) / i) % 4.0 * 90.0), z.append(za * rng.choice([-1.0, 1.0], n))
    # the polar / equatorial boundary and the azimuth seam
    k = 200
    z.append(np.concatenate([2.0 / 3.0 + rng.choice(offs, k), -2.0 / 3.0 + rng.choice(offs, k)]))
    ra.append(rng.uniform(0, 360, 2 * k))
    z.append(rng.uniform(-1, 1, 2 * k))
    ra.append(np.concatenate([rng.choice(offs, k) * 90.0, 360.0 + rng.choice(offs, k) * 90.0]))
    ra = np.concatenate(ra)
    z = np.clip(np.concatenate(z), -1.0, 1.0)
    ra = ra + 360.0 * rng.integers(-1, 2, ra.size)          # wrap in both directions
    return ra, np.degrees(np.arcsin(z))
