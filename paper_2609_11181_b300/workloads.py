"""Seeded synthetic workloads at the benchmark configurations.

Each builder returns device tensors ready for the C ABI.  The input model is
the one of ``synth`` (SIS halo fields + shape noise on spherical caps); the
shapes, densities and scales are the stated configurations:

  pixel4096  15,000 deg^2 cap at (0, 0); binned shear at NSIDE 4096 with
             Poisson(22) counts per pixel; Poisson field of 20,000 SIS
             (theta_E log-uniform 0.1-1.5'); output NSIDE 4096 over the
             footprint; Schirmer filter x_c = 0.15, theta_ap = 10'.
  brute2048  1,000 deg^2 cap; 5e7 galaxies, half in Gaussian clumps of 1'
             (20 per clump), w ~ U[0.5, 1.5]; same SIS density; sorted
             into NSIDE 4096; output NSIDE 2048; polynomial filter, 15'.
  c1         10 deg cap at (0, 0); 2e5 uniform galaxies, 5 SIS
             (theta_E 0.2-1'); output NSIDE 256; polynomial, 60'.

Pixel centres for the binned field come from the caller (``centres_fn``):
the benchmark passes the library's device pix2vec, the tests pass the
float64 oracle's.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import synth

ARCMIN = math.pi / 10800.0
HALO_DENSITY = 20000.0 / 15000.0          # SIS per deg^2
SIS_TRUNC = math.radians(1.0)             # each SIS contributes within 1 deg


@dataclass
class PixelWorkload:
    nside: int
    theta_ap_arcmin: float
    filter: str
    targets: torch.Tensor          # int64 RING pixels (device)
    G1: torch.Tensor
    G2: torch.Tensor
    W: torch.Tensor
    S2: torch.Tensor
    n: torch.Tensor                # int32
    n_halos: int
    desc: str


@dataclass
class GalaxyWorkload:
    nside_out: int
    nside_bin: int
    theta_ap_arcmin: float
    filter: str
    targets: torch.Tensor
    cat: synth.Catalog
    n_halos: int
    desc: str


def _cap_mask(centres: torch.Tensor, ra0: float, dec0: float, radius: float) -> torch.Tensor:
    a, d = math.radians(ra0), math.radians(dec0)
    axis = torch.tensor([math.cos(d) * math.cos(a), math.cos(d) * math.sin(a), math.sin(d)],
                        dtype=centres.dtype, device=centres.device)
    return (centres @ axis) >= math.cos(radius)


def all_centres(nside: int, centres_fn, device, chunk: int = 1 << 25) -> torch.Tensor:
    npix = 12 * nside * nside
    out = torch.empty((npix, 3), dtype=torch.float64, device=device)
    for s in range(0, npix, chunk):
        p = torch.arange(s, min(npix, s + chunk), dtype=torch.int64, device=device)
        out[s:s + p.numel()] = centres_fn(nside, p)
    return out


def pixel_workload(device, centres_fn, nside=4096, area_deg2=15000.0, mean_count=22.0, theta_ap=10.0,
                   filt="schirmer", seed=2609, ra0=0.0, dec0=0.0) -> PixelWorkload:
    gen = synth.make_gen(seed, device)
    radius = synth.cap_radius_for_area(area_deg2)
    v = all_centres(nside, centres_fn, device)
    foot = _cap_mask(v, ra0, dec0, radius)
    halos = synth.halos_poisson(HALO_DENSITY, area_deg2, ra0, dec0, radius, gen)
    b = synth.binned_field(v, foot, mean_count, halos, gen, r_trunc=SIS_TRUNC)
    del v
    targets = torch.nonzero(foot, as_tuple=False).flatten().to(torch.int64)
    desc = (f"{area_deg2:.0f} deg^2 cap at ({ra0},{dec0}); binned NSIDE {nside}, Poisson({mean_count}) "
            f"counts; {halos.ra_deg.numel()} SIS; output NSIDE {nside}; {filt} theta_ap={theta_ap}'")
    return PixelWorkload(nside, theta_ap, filt, targets, b.G1, b.G2, b.W, b.S2, b.n, halos.ra_deg.numel(), desc)


def galaxy_workload(device, centres_fn, n_gal=50_000_000, area_deg2=1000.0, nside_bin=4096, nside_out=2048,
                    theta_ap=15.0, filt="poly", seed=2610, ra0=0.0, dec0=0.0, clumped=True,
                    w_range=(0.5, 1.5)) -> GalaxyWorkload:
    gen = synth.make_gen(seed, device)
    radius = synth.cap_radius_for_area(area_deg2)
    halos = synth.halos_poisson(HALO_DENSITY, area_deg2, ra0, dec0, radius, gen)
    cat = synth.galaxy_catalog(n_gal, ra0, dec0, radius, halos, gen, r_trunc=SIS_TRUNC, clumped=clumped,
                               w_range=w_range)
    v = all_centres(nside_out, centres_fn, device)
    targets = torch.nonzero(_cap_mask(v, ra0, dec0, radius), as_tuple=False).flatten().to(torch.int64)
    desc = (f"{area_deg2:.0f} deg^2 cap; {n_gal} galaxies ({'half clumped' if clumped else 'uniform'}), "
            f"w~U{w_range}; {halos.ra_deg.numel()} SIS; bins NSIDE {nside_bin}; output NSIDE {nside_out}; "
            f"{filt} theta_ap={theta_ap}'")
    return GalaxyWorkload(nside_out, nside_bin, theta_ap, filt, targets, cat, halos.ra_deg.numel(), desc)


def c1_workload(device, centres_fn, seed=101) -> GalaxyWorkload:
    gen = synth.make_gen(seed, device)
    radius = math.radians(10.0)
    halos = synth.halos_uniform(5, 0.0, 0.0, radius, gen, 0.2 * ARCMIN, 1.0 * ARCMIN)
    cat = synth.galaxy_catalog(200_000, 0.0, 0.0, radius, halos, gen, r_trunc=math.radians(2.0))
    v = all_centres(256, centres_fn, device)
    targets = torch.nonzero(_cap_mask(v, 0.0, 0.0, radius), as_tuple=False).flatten().to(torch.int64)
    return GalaxyWorkload(256, 1024, 60.0, "poly", targets, cat, 5,
                          "10 deg cap; 2e5 uniform galaxies; 5 SIS; output NSIDE 256; poly 60'")


# the benchmark configurations (keyword arguments of the builders above)
PIXEL_WORKLOADS = {
    # the headline configuration
    "pixel4096": dict(nside=4096, area_deg2=15000.0, theta_ap=10.0, filt="schirmer"),
    # a small case of the same kernels for profiling: 3,000 deg^2 cap at dec 60
    # (polar and equatorial rings), NSIDE 2048, theta_ap = 20' (about as many
    # pixels per aperture as NSIDE 4096 at 10'); 1 GB of full-sky arrays
    "pixel2048": dict(nside=2048, area_deg2=3000.0, theta_ap=20.0, filt="schirmer", dec0=60.0),
    # the same at the equator (Toeplitz kernel only)
    "pixel2048eq": dict(nside=2048, area_deg2=3000.0, theta_ap=20.0, filt="schirmer", dec0=0.0),
}

GALAXY_WORKLOADS = {
    # 5e7 clustered galaxies on a 1,000 deg^2 cap, sorted into NSIDE 4096,
    # output NSIDE 2048, polynomial filter, 15'
    "brute2048": dict(n_gal=50_000_000, area_deg2=1000.0, nside_bin=4096, nside_out=2048, theta_ap=15.0,
                      filt="poly"),
    # a small case of the same kernels for profiling
    "brute_small": dict(n_gal=4_000_000, area_deg2=100.0, nside_bin=4096, nside_out=2048, theta_ap=15.0,
                        filt="poly"),
}
