"""Seeded synthetic inputs for the aperture-mass workloads.

This module holds only the *input model* -- where galaxies sit, what shear
they carry -- and none of the aperture-mass method itself (no pixelisation,
no aperture sums, no filters).  Both the CUDA path and the FP64 oracle are
fed from here; it imports neither.

Input model (stands in for the paper's Takahashi+2017 / HSC-Y3 mock of
Sect. 4, which is not available):
  * positions uniform on a spherical cap, optionally half of them in
    Gaussian clumps (a Thomas process) for clustered catalogues;
  * shear = sum of singular isothermal spheres (SIS), gamma_t = theta_E /
    (2 theta), truncated at ``r_trunc``, written in the local (East, North)
    basis with gamma_t > 0 meaning tangential alignment;
  * Gaussian shape noise, sigma_e = 0.26 per component (Sect. 6);
  * binned maps (pixel-based workloads) get Poisson counts per pixel and a
    mean shear = signal + N(0, sigma_e^2 / n).

All functions run on whatever device the given torch generator lives on, so
the same code makes the small CPU test cases and the full-size GPU bench
inputs.  Angles are radians unless a name says ``_deg``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

ARCMIN = math.pi / (180.0 * 60.0)
DEG = math.pi / 180.0
SIGMA_E = 0.26


def make_gen(seed: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def cap_radius_for_area(area_deg2: float) -> float:
    """Radius (rad) of the spherical cap of the given area: 1 - cos r = A / 2pi."""
    a = area_deg2 * DEG * DEG
    return math.acos(1.0 - a / (2.0 * math.pi))


def _rot_to(ra0: float, dec0: float, x, y, z):
    """Rotate vectors given about the +z axis so that +z lands on (ra0, dec0)."""
    # first tilt about y by (90 deg - dec0), then spin about z by ra0
    t = math.pi / 2 - dec0
    ct, st = math.cos(t), math.sin(t)
    x1 = ct * x + st * z
    z1 = -st * x + ct * z
    ca, sa = math.cos(ra0), math.sin(ra0)
    return ca * x1 - sa * y, sa * x1 + ca * y, z1


def vec_to_radec_deg(x, y, z):
    ra = torch.rad2deg(torch.atan2(y, x)) % 360.0
    dec = torch.rad2deg(torch.asin(torch.clamp(z, -1.0, 1.0)))
    return ra, dec


def radec_deg_to_vec(ra, dec):
    a, d = torch.deg2rad(ra), torch.deg2rad(dec)
    cd = torch.cos(d)
    return torch.stack([cd * torch.cos(a), cd * torch.sin(a), torch.sin(d)], dim=-1)


def uniform_cap(n: int, ra0_deg: float, dec0_deg: float, radius: float,
                gen: torch.Generator, dtype=torch.float64):
    """n points uniform on the sphere inside a cap; returns (ra_deg, dec_deg)."""
    dev = gen.device
    u = torch.rand(n, generator=gen, device=dev, dtype=dtype)
    v = torch.rand(n, generator=gen, device=dev, dtype=dtype)
    z = 1.0 - u * (1.0 - math.cos(radius))
    phi = 2.0 * math.pi * v
    r = torch.sqrt(torch.clamp((1.0 - z) * (1.0 + z), min=0.0))
    x, y = r * torch.cos(phi), r * torch.sin(phi)
    x, y, z = _rot_to(math.radians(ra0_deg), math.radians(dec0_deg), x, y, z)
    return vec_to_radec_deg(x, y, z)


def clumpy_cap(n: int, ra0_deg: float, dec0_deg: float, radius: float,
               gen: torch.Generator, frac_clumped: float = 0.5,
               clump_sigma: float = 1.0 * ARCMIN, per_clump: int = 20):
    """Thomas process: a fraction of the points in Gaussian clumps, the rest uniform."""
    n_cl = int(round(n * frac_clumped)) // per_clump * per_clump
    n_un = n - n_cl
    ra_u, dec_u = uniform_cap(n_un, ra0_deg, dec0_deg, radius, gen)
    if n_cl == 0:
        return ra_u, dec_u
    k = n_cl // per_clump
    rac, decc = uniform_cap(k, ra0_deg, dec0_deg, radius * 0.98, gen)
    dev = gen.device
    # offsets in the local tangent plane of each clump centre
    dx = torch.randn(n_cl, generator=gen, device=dev, dtype=torch.float64) * clump_sigma
    dy = torch.randn(n_cl, generator=gen, device=dev, dtype=torch.float64) * clump_sigma
    c = radec_deg_to_vec(rac, decc).repeat_interleave(per_clump, dim=0)
    a = torch.deg2rad(rac).repeat_interleave(per_clump)
    d = torch.deg2rad(decc).repeat_interleave(per_clump)
    east = torch.stack([-torch.sin(a), torch.cos(a), torch.zeros_like(a)], -1)
    north = torch.stack([-torch.sin(d) * torch.cos(a), -torch.sin(d) * torch.sin(a), torch.cos(d)], -1)
    p = c + dx[:, None] * east + dy[:, None] * north
    p = p / torch.linalg.norm(p, dim=-1, keepdim=True)
    ra_c, dec_c = vec_to_radec_deg(p[:, 0], p[:, 1], p[:, 2])
    return torch.cat([ra_u, ra_c]), torch.cat([dec_u, dec_c])


@dataclass
class Halos:
    ra_deg: torch.Tensor
    dec_deg: torch.Tensor
    theta_e: torch.Tensor          # Einstein radius, rad


def halos_uniform(k: int, ra0_deg, dec0_deg, radius, gen, te_lo, te_hi, log=False) -> Halos:
    ra, dec = uniform_cap(k, ra0_deg, dec0_deg, radius, gen)
    u = torch.rand(k, generator=gen, device=gen.device, dtype=torch.float64)
    if log:
        te = torch.exp(math.log(te_lo) + u * (math.log(te_hi) - math.log(te_lo)))
    else:
        te = te_lo + u * (te_hi - te_lo)
    return Halos(ra, dec, te)


def halos_poisson(density_per_deg2: float, area_deg2: float, ra0_deg, dec0_deg, radius,
                  gen, te_lo=0.1 * ARCMIN, te_hi=1.5 * ARCMIN) -> Halos:
    lam = torch.tensor([density_per_deg2 * area_deg2], dtype=torch.float64, device=gen.device)
    k = int(torch.poisson(lam, generator=gen).item())
    return halos_uniform(k, ra0_deg, dec0_deg, radius, gen, te_lo, te_hi, log=True)


def sis_shear(ra_deg, dec_deg, halos: Halos, r_trunc: float, chunk: int = 1 << 21, inner_cut: bool = True):
    """Summed SIS shear (gamma_1, gamma_2) in the local (East, North) basis.

    gamma_t = theta_E / (2 theta) for 0 < theta <= r_trunc; with inner_cut
    the strong-lensing core theta < theta_E is held at gamma_t = 1/2.  The orientation
    uses the great-circle bearing b of the halo seen from the point (from
    North through East): gamma_1 = gamma_t cos 2b, gamma_2 = -gamma_t sin 2b,
    so a point East of a halo is stretched North-South (gamma_1 < 0).

    Halos are bucketed on a cubic grid of cell size 2 * chord(r_trunc); each
    point looks at the 8 cells around it, which contain every halo within
    r_trunc.
    """
    dev = ra_deg.device
    n = ra_deg.numel()
    g1 = torch.zeros(n, dtype=torch.float64, device=dev)
    g2 = torch.zeros(n, dtype=torch.float64, device=dev)
    if halos.ra_deg.numel() == 0 or n == 0:
        return g1, g2
    hv = radec_deg_to_vec(halos.ra_deg.to(dev), halos.dec_deg.to(dev))
    hte = halos.theta_e.to(dev)
    ha, hd = torch.deg2rad(halos.ra_deg.to(dev)), torch.deg2rad(halos.dec_deg.to(dev))
    L = 2.0 * 2.0 * math.sin(0.5 * r_trunc) * 1.0001
    nc = int(math.ceil(2.0 / L)) + 3
    hc = torch.floor((hv + 1.0) / L).long() + 1

    def key(c):
        return (c[..., 0] * nc + c[..., 1]) * nc + c[..., 2]

    hk = key(hc)
    order = torch.argsort(hk)
    hk_s = hk[order]
    uniq, counts = torch.unique_consecutive(hk_s, return_counts=True)
    maxc = int(counts.max().item())
    starts = torch.cumsum(counts, 0) - counts
    table = torch.full((uniq.numel(), maxc), -1, dtype=torch.long, device=dev)
    slot = torch.arange(hk_s.numel(), device=dev) - torch.repeat_interleave(starts, counts)
    cell_of = torch.repeat_interleave(torch.arange(uniq.numel(), device=dev), counts)
    table[cell_of, slot] = order
    cos_tr = math.cos(r_trunc)
    corners = torch.tensor([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)],
                           dtype=torch.long, device=dev)
    for s in range(0, n, chunk):
        ra = torch.deg2rad(ra_deg[s:s + chunk])
        dec = torch.deg2rad(dec_deg[s:s + chunk])
        m = ra.numel()
        ca, sa, cd, sd = torch.cos(ra), torch.sin(ra), torch.cos(dec), torch.sin(dec)
        pv = torch.stack([cd * ca, cd * sa, sd], -1)
        base = torch.floor((pv + 1.0) / L - 0.5).long() + 1
        cells = base[:, None, :] + corners[None, :, :]          # (m, 8, 3)
        ck = key(cells)
        pos = torch.searchsorted(uniq, ck.reshape(-1)).clamp(max=uniq.numel() - 1)
        hit = uniq[pos] == ck.reshape(-1)
        cand = table[pos]                                       # (m*8, maxc)
        cand = torch.where(hit[:, None], cand, torch.full_like(cand, -1))
        cand = cand.reshape(m, 8 * maxc)
        ci = cand.clamp(min=0)
        cosd = pv[:, 0:1] * hv[ci, 0] + pv[:, 1:2] * hv[ci, 1] + pv[:, 2:3] * hv[ci, 2]
        rows, cols = torch.nonzero((cand >= 0) & (cosd >= cos_tr), as_tuple=True)
        hi = ci[rows, cols]
        h = hv[hi]
        # separation from the chord; bearing b of the halo from the point (from
        # North through East) from its components along the local East and North
        theta = 2.0 * torch.asin(torch.clamp(0.5 * torch.linalg.norm(h - pv[rows], dim=-1), max=1.0))
        te = hte[hi]
        th_eff = torch.maximum(theta, te) if inner_cut else torch.clamp(theta, min=1e-30)
        gt = torch.where(theta > 0, te / (2.0 * th_eff), torch.zeros_like(theta))
        a_c, a_s, d_c, d_s = ca[rows], sa[rows], cd[rows], sd[rows]
        eh = -a_s * h[:, 0] + a_c * h[:, 1]                    # sin(b) * sin(theta)
        nh = -d_s * (a_c * h[:, 0] + a_s * h[:, 1]) + d_c * h[:, 2]  # cos(b) * sin(theta)
        q = eh * eh + nh * nh
        qs = torch.where(q > 0, q, torch.ones_like(q))
        c2b = torch.where(q > 0, (nh * nh - eh * eh) / qs, torch.ones_like(q))
        s2b = torch.where(q > 0, 2.0 * eh * nh / qs, torch.zeros_like(q))
        # back to one row per point (unique positions) and summed in a fixed order
        t1 = torch.zeros((m, 8 * maxc), dtype=torch.float64, device=dev)
        t2 = torch.zeros((m, 8 * maxc), dtype=torch.float64, device=dev)
        t1[rows, cols] = gt * c2b
        t2[rows, cols] = -gt * s2b
        g1[s:s + chunk] = t1.sum(-1)
        g2[s:s + chunk] = t2.sum(-1)
    return g1, g2


@dataclass
class Catalog:
    ra_deg: torch.Tensor    # float64
    dec_deg: torch.Tensor   # float64
    e1: torch.Tensor        # float32
    e2: torch.Tensor        # float32
    w: torch.Tensor         # float32

    def to(self, device):
        return Catalog(*(getattr(self, k).to(device) for k in ("ra_deg", "dec_deg", "e1", "e2", "w")))

    @property
    def n(self):
        return self.ra_deg.numel()


def galaxy_catalog(n: int, ra0_deg: float, dec0_deg: float, radius: float, halos: Halos,
                   gen: torch.Generator, r_trunc: float, clumped: bool = False,
                   w_range=None, sigma_e: float = SIGMA_E) -> Catalog:
    if clumped:
        ra, dec = clumpy_cap(n, ra0_deg, dec0_deg, radius, gen)
    else:
        ra, dec = uniform_cap(n, ra0_deg, dec0_deg, radius, gen)
    g1, g2 = sis_shear(ra, dec, halos, r_trunc)
    dev = gen.device
    e1 = g1 + sigma_e * torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
    e2 = g2 + sigma_e * torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
    if w_range is None:
        w = torch.ones(n, dtype=torch.float32, device=dev)
    else:
        u = torch.rand(n, generator=gen, device=dev, dtype=torch.float64)
        w = (w_range[0] + u * (w_range[1] - w_range[0])).float()
    return Catalog(ra, dec, e1.float(), e2.float(), w)


@dataclass
class Binned:
    """Full-sky per-pixel sums on a RING grid (zeros outside the footprint)."""
    G1: torch.Tensor     # float32, sum w e1
    G2: torch.Tensor     # float32, sum w e2
    W: torch.Tensor      # float32, sum w
    S2: torch.Tensor     # float32, sum w^2 |e|^2
    n: torch.Tensor      # int32 count


def binned_field(centres: torch.Tensor, in_footprint: torch.Tensor, mean_count: float,
                 halos: Halos, gen: torch.Generator, r_trunc: float,
                 sigma_e: float = SIGMA_E, chunk: int = 1 << 24) -> Binned:
    """Per-pixel binned shear at given pixel-centre unit vectors.

    n_p ~ Poisson(mean_count) inside the footprint; G_p = n_p (gamma_SIS(p) +
    N(0, sigma_e^2 / n_p)) per component; W_p = n_p;
    S2_p = n_p (2 sigma_e^2 + |gamma_SIS(p)|^2).  The caller supplies the
    centres (any HEALPix implementation) and the footprint mask.
    """
    dev = centres.device
    npix = centres.shape[0]
    G1 = torch.zeros(npix, dtype=torch.float32, device=dev)
    G2 = torch.zeros_like(G1)
    W = torch.zeros_like(G1)
    S2 = torch.zeros_like(G1)
    cnt = torch.zeros(npix, dtype=torch.int32, device=dev)
    idx = torch.nonzero(in_footprint, as_tuple=False).flatten()
    for s in range(0, idx.numel(), chunk):
        ii = idx[s:s + chunk]
        v = centres[ii].to(torch.float64)
        ra, dec = vec_to_radec_deg(v[:, 0], v[:, 1], v[:, 2])
        lam = torch.full((ii.numel(),), float(mean_count), dtype=torch.float64, device=dev)
        n = torch.poisson(lam, generator=gen)
        g1, g2 = sis_shear(ra, dec, halos, r_trunc)
        nz = torch.clamp(n, min=1.0)
        sd = sigma_e / torch.sqrt(nz)
        m1 = g1 + sd * torch.randn(ii.numel(), generator=gen, device=dev, dtype=torch.float64)
        m2 = g2 + sd * torch.randn(ii.numel(), generator=gen, device=dev, dtype=torch.float64)
        G1[ii] = (n * m1).float()
        G2[ii] = (n * m2).float()
        W[ii] = n.float()
        S2[ii] = (n * (2 * sigma_e ** 2 + g1 * g1 + g2 * g2)).float()
        cnt[ii] = n.to(torch.int32)
    return Binned(G1, G2, W, S2, cnt)


# ---------------------------------------------------------------------------
# random draws of the learned correction (passed to both sides as inputs)
# ---------------------------------------------------------------------------
MLP_LAYERS = ((64, 4), (64, 64), (1, 64))      # (out, in) of the three linear layers


def mlp_init_params(seed: int) -> torch.Tensor:
    """Initial parameter vector of the 4 -> 64 -> 64 -> 1 network (float32, CPU).

    Layout W1 [64][4], b1 [64], W2 [64][64], b2 [64], w3 [64], b3; every
    weight and bias of a layer uniform in +-1/sqrt(fan_in)."""
    g = make_gen(seed)
    parts_w, parts_b = [], []
    for out, fan_in in MLP_LAYERS:
        bound = 1.0 / math.sqrt(fan_in)
        parts_w.append((torch.rand(out * fan_in, generator=g, dtype=torch.float64) * 2 - 1) * bound)
        parts_b.append((torch.rand(out, generator=g, dtype=torch.float64) * 2 - 1) * bound)
    return torch.cat([parts_w[0], parts_b[0], parts_w[1], parts_b[1], parts_w[2], parts_b[2]]).float()


def minibatches(n: int, batch: int, epochs: int, seed: int, device="cpu"):
    """Shuffled minibatch index lists (int32) for ``epochs`` passes over n samples."""
    g = make_gen(seed, device)
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g, device=device).to(torch.int32)
        for s in range(0, n - batch + 1, batch):
            yield perm[s:s + batch]
