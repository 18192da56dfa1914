"""GPU parity of the aperture-mass maps against the float64 oracle.

Bar: member counts bit-exact; per map rms(M_gpu - M_oracle)/rms(M_oracle)
<= 1e-4 for M_E, M_B and sigma^2 (the float32 accumulation tolerance the
design states); weight sums within 1e-6 relative.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2609_11181_b300 import api

from _cases import ARCMIN, binned_field_oracle, c1_catalog, cap_targets, catalog, rms_rel

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _check(got, ref, label=""):
    np.testing.assert_array_equal(got["count"].cpu().numpy(), ref["N"], err_msg=label + " counts")
    sw = got["sum_w"].cpu().numpy()
    np.testing.assert_allclose(sw, ref["SW"], rtol=1e-6, atol=1e-12, err_msg=label + " sum_w")
    for k_got, k_ref in (("map_e", "ME"), ("map_b", "MB"), ("var", "VAR")):
        e = rms_rel(got[k_got].cpu().numpy(), ref[k_ref])
        assert e <= TOL, f"{label} {k_got}: rms rel err {e:.3e}"


def _gal_run(dev, cat, targets, nside_out, nside_bin, theta_arcmin, filt, xc=0.15):
    ctx = api.Context(nside_out, theta_arcmin, filt, xc=xc, nside_bin=nside_bin)
    c = cat.to(dev)
    ctx.set_targets(torch.from_numpy(targets).to(dev))
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    bf = ctx.map_bruteforce()
    nbf = None
    ctx.sync(120)
    nbf = ctx.fp64_decisions()
    px = ctx.map_pixel()
    ctx.sync(120)
    return ctx, bf, px, nbf


def _oracle_maps(cat, targets, nside_out, nside_bin, theta_arcmin, kind, xc=0.15):
    th = theta_arcmin * ARCMIN
    cv = oracle.pix2vec(nside_out, targets)
    ra, dec = cat.ra_deg.numpy(), cat.dec_deg.numpy()
    e1, e2, w = cat.e1.double().numpy(), cat.e2.double().numpy(), cat.w.double().numpy()
    bf = oracle.map_galaxies(cv, ra, dec, e1, e2, w, kind, th, xc)
    b = oracle.bin_catalog(nside_bin, ra, dec, e1, e2, w)
    px = oracle.map_pixels(cv, nside_bin, b["G1"], b["G2"], b["W"], b["S2"], b["n"], kind, th, xc)
    return bf, px


def test_c1_config(cuda_device):
    """Config C1: NSIDE 256 in a 10 deg cap, 200k galaxies, 5 SIS, polynomial, 60'."""
    cat = c1_catalog()
    tg = cap_targets(256, 0.0, 0.0, 10.0)
    ctx, bf, px, nfp = _gal_run(cuda_device, cat, tg, 256, 1024, 60.0, "poly")
    rbf, rpx = _oracle_maps(cat, tg, 256, 1024, 60.0, 1)
    _check(bf, rbf, "brute")
    _check(px, rpx, "pixel")
    assert nfp < 0.05 * len(tg) * 10


@pytest.mark.parametrize("ra0,dec0,rad,no,nb,th,filt", [
    (40.0, 70.0, 5.0, 512, 512, 10.0, "schirmer"),     # crosses the polar/equatorial boundary
    (300.0, 89.3, 2.5, 256, 256, 40.0, "poly"),        # around the north pole (whole, wide rings)
    (120.0, -88.0, 3.0, 128, 512, 30.0, "schirmer"),   # south pole, nside_out != nside_bin
    (359.5, -30.0, 4.0, 128, 256, 25.0, "poly"),       # RA wrap at 0/360
    (10.0, 0.0, 2.0, 1024, 1024, 5.0, "schirmer"),     # equator, small aperture
])
def test_maps_geometry_cases(cuda_device, ra0, dec0, rad, no, nb, th, filt):
    kind = 1 if filt == "poly" else 2
    cat = catalog(int(ra0 * 7 + dec0 * 3 + 1000), 60_000, ra0, dec0, rad + th / 60.0, nhalo=6,
                  w_range=(0.5, 1.5), clumped=True)
    tg = cap_targets(no, ra0, dec0, rad)
    ctx, bf, px, _ = _gal_run(cuda_device, cat, tg, no, nb, th, filt)
    rbf, rpx = _oracle_maps(cat, tg, no, nb, th, kind)
    _check(bf, rbf, "brute")
    _check(px, rpx, "pixel")


@pytest.mark.parametrize("th", [150.0, 300.0])
def test_toeplitz_run_lengths(cuda_device, th):
    """Equatorial rings at NSIDE 512 (6.9' pixels): a 150' aperture gives
    Toeplitz runs of about 45 offsets (the 64-offset staging), a 300'
    aperture runs of about 90 (the 120-offset staging)."""
    ra0, dec0, rad = 10.0, 0.0, 2.0
    cat = catalog(4242 + int(th), 120_000, ra0, dec0, rad + th / 60.0 + 0.5, nhalo=8, w_range=(0.5, 1.5))
    tg = cap_targets(512, ra0, dec0, rad)
    ctx, bf, px, _ = _gal_run(cuda_device, cat, tg, 512, 512, th, "schirmer")
    assert ctx.general_targets().numel() < len(tg) // 4       # most targets on Toeplitz rings
    rbf, rpx = _oracle_maps(cat, tg, 512, 512, th, 2)
    _check(px, rpx, f"pixel {th}'")
    _check(bf, rbf, f"brute {th}'")


@pytest.mark.parametrize("th", [30.0, 300.0])
def test_brute_force_members_at_the_band_edges(cuda_device, th):
    """Galaxies placed at chord^2 = T (1 + r) from a target, with r stepping
    by 2e-9 (a few hundredths of a float32 ulp) across both edges of the
    float32 guard band (r = -+4e-6) and across T itself: every pair is
    decided as the float64 definition decides it, so the member counts equal
    the oracle's."""
    nside = 256
    T = api.chord2(th)
    tg = cap_targets(nside, 30.0, 20.0, 1.5)[:40]
    cv = oracle.pix2vec(nside, tg)
    rng = np.random.default_rng(5)
    rel = np.concatenate([c + 2e-9 * np.arange(-40, 41) for c in (-4e-6, 0.0, 4e-6)])
    pts = []
    for t in cv:
        e = np.cross([0.0, 0.0, 1.0], t)
        e /= np.linalg.norm(e)
        n = np.cross(t, e)
        d = 2.0 * np.arcsin(0.5 * np.sqrt(T * (1.0 + rel)))
        b = rng.uniform(0.0, 2.0 * math.pi, rel.size)
        v = (np.cos(d)[:, None] * t + np.sin(d)[:, None] * (np.cos(b)[:, None] * n + np.sin(b)[:, None] * e))
        pts.append(v)
    v = np.concatenate(pts)
    ra = np.degrees(np.arctan2(v[:, 1], v[:, 0])) % 360.0
    dec = np.degrees(np.arcsin(np.clip(v[:, 2], -1.0, 1.0)))
    ng = ra.size
    e1 = rng.normal(0.0, 0.2, ng)
    e2 = rng.normal(0.0, 0.2, ng)
    w = rng.uniform(0.5, 1.5, ng)
    ref = oracle.map_galaxies(cv, ra, dec, e1, e2, w, 1, th * ARCMIN)
    dev = cuda_device
    ctx = api.Context(nside, th, "poly", nside_bin=1024)
    ctx.set_targets(torch.from_numpy(tg).to(dev))
    ctx.bin_galaxies(torch.from_numpy(ra).to(dev), torch.from_numpy(dec).to(dev),
                     torch.from_numpy(e1).float().to(dev), torch.from_numpy(e2).float().to(dev),
                     torch.from_numpy(w).float().to(dev))
    got = ctx.map_bruteforce()
    ctx.sync(60)
    np.testing.assert_array_equal(got["count"].cpu().numpy(), ref["N"])
    assert ctx.fp64_decisions() > 0
    ctx.close()


@pytest.mark.parametrize("no,nb,th,filt,rad", [
    (1024, 8192, 8.0, "poly", 1.0),      # fine bins: many short bin rings per output ring
    (64, 256, 300.0, "poly", 3.0),       # a 5 degree aperture: the four-term series and the
                                         # polynomial weight's d^2 / sin^2 d terms beyond the first
])
def test_maps_bin_and_aperture_extremes(cuda_device, no, nb, th, filt, rad):
    ra0, dec0 = 140.0, -25.0
    cat = catalog(int(th * 10) + nb, 150_000, ra0, dec0, rad + th / 60.0 + 0.5, nhalo=6, w_range=(0.5, 1.5),
                  clumped=True)
    tg = cap_targets(no, ra0, dec0, rad)
    ctx, bf, px, _ = _gal_run(cuda_device, cat, tg, no, nb, th, filt)
    rbf, rpx = _oracle_maps(cat, tg, no, nb, th, 1)
    _check(bf, rbf, f"brute {no}/{nb}/{th}'")
    _check(px, rpx, f"pixel {no}/{nb}/{th}'")
    ctx.close()


def test_general_mirror_pairs(cuda_device):
    """General targets whose mirror image about a meridian m pi/4 is a target
    too run in pairs that share each pair's geometry.  The cap is centred on
    the meridian pi/4 at polar ring 20 of NSIDE 64 with the aperture of the
    in-place test below (every target of ring 20 has guard-band pairs), so
    nearly every general target is paired and the images' guard-band pairs
    are decided from the shared window.  Checked: the pairs are mirror images
    (one ring, azimuths summing to a multiple of pi/2) and disjoint; the map
    against the oracle; one slot (images finished in place) bit-identical."""
    nside, ring = 64, 20
    z = 1.0 - ring * ring / (3.0 * nside * nside)
    rho = math.sqrt((1.0 - z) * (1.0 + z))
    theta_arcmin = 2.0 * math.asin(rho * math.sin(3 * (2 * math.pi / (4 * ring)) / 2)) / ARCMIN
    dec_ring = math.degrees(math.asin(z))
    cat = catalog(24, 60_000, 45.0, dec_ring, 8.0, w_range=(0.5, 1.5))
    tg = cap_targets(nside, 45.0, dec_ring, 5.0)
    dev = cuda_device
    ctx = api.Context(nside, theta_arcmin, "schirmer", nside_bin=nside)
    c = cat.to(dev)
    ctx.set_targets(torch.from_numpy(tg).to(dev))
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    a = ctx.map_pixel()
    ctx.sync(60)
    pairs, n_single = ctx.general_pairs()
    gen = ctx.general_targets().cpu().numpy()
    p = pairs.cpu().numpy()
    assert 2 * len(p) + n_single == len(gen)
    assert len(p) >= 0.4 * len(gen)
    flat = p.ravel()
    assert np.unique(flat).size == flat.size and np.isin(flat, gen).all()
    v = oracle.pix2vec(nside, tg[flat]).reshape(-1, 2, 3)
    assert np.array_equal(v[:, 0, 2], v[:, 1, 2])
    phi = np.arctan2(v[..., 1], v[..., 0])
    q = (phi[:, 0] + phi[:, 1]) / (math.pi / 2)
    assert np.abs(q - np.round(q)).max() < 1e-9
    on_ring = [i for i in flat if oracle.pix_info(nside, int(tg[i]))[0] == ring]
    assert len(on_ring) >= 8
    _, rpx = _oracle_maps(cat, tg, nside, nside, theta_arcmin, 2)
    _check(a, rpx, "mirror pairs")
    n_fp64 = ctx.fp64_decisions()
    assert n_fp64 >= 2 * len(on_ring)
    ctx.set_band_slot_limit(1)
    b = ctx.map_pixel()
    ctx.sync(60)
    assert ctx.fp64_decisions() == n_fp64
    for k in ("map_e", "map_b", "var", "sum_w", "count", "members"):
        assert torch.equal(a[k], b[k]), k
    ctx.close()


def test_pixel_mode_binned_field(cuda_device):
    """Pixel-based workload shape (Poisson counts, SIS field) at nside 512, Schirmer 10'."""
    nside = 512
    b, foot = binned_field_oracle(5, nside, 0.0, 30.0, 6.0, mean_count=22.0)
    tg = np.nonzero(foot)[0].astype(np.int64)
    dev = cuda_device
    ctx = api.Context(nside, 10.0, "schirmer", nside_bin=nside)
    ctx.set_targets(torch.from_numpy(tg).to(dev))
    ctx.set_binned(*(x.to(dev) for x in (b.G1, b.G2, b.W, b.S2, b.n)))
    got = ctx.map_pixel()
    ctx.sync(60)
    ref = oracle.map_pixels(oracle.pix2vec(nside, tg), nside, b.G1.double().numpy(), b.G2.double().numpy(),
                            b.W.double().numpy(), b.S2.double().numpy(), b.n.long().numpy(), 2, 10.0 * ARCMIN)
    _check(got, ref, "binned")


def test_zero_shear_and_empty_targets(cuda_device):
    cat = catalog(3, 20_000, 80.0, 20.0, 3.0)
    cat.e1.zero_()
    cat.e2.zero_()
    tg = cap_targets(128, 80.0, 20.0, 2.0)
    ctx, bf, px, _ = _gal_run(cuda_device, cat, tg, 128, 256, 20.0, "poly")
    for m in (bf, px):
        assert float(m["map_e"].abs().max()) == 0.0 and float(m["map_b"].abs().max()) == 0.0
        assert float(m["var"].abs().max()) == 0.0
    ctx.set_targets(torch.empty(0, dtype=torch.int64, device=cuda_device))
    out = ctx.map_pixel()
    ctx.sync(10)
    assert out["map_e"].numel() == 0


def test_targets_outside_footprint(cuda_device):
    # targets far from every galaxy: zero weight, zero maps, zero counts
    cat = catalog(4, 5000, 10.0, 10.0, 1.0)
    tg = cap_targets(64, 190.0, -10.0, 3.0)
    ctx, bf, px, _ = _gal_run(cuda_device, cat, tg, 64, 64, 10.0, "poly")
    for m in (bf, px):
        assert int(m["count"].sum()) == 0 and float(m["sum_w"].abs().sum()) == 0.0


def test_packed_and_soa_inputs_agree(cuda_device):
    # smart_set_binned (copied into the packed layout) and smart_set_binned_packed
    # (borrowed) give identical maps; smart_get_binned returns the arrays given
    nside = 128
    b, foot = binned_field_oracle(9, nside, 200.0, -40.0, 10.0, mean_count=15.0)
    tg = torch.from_numpy(np.nonzero(foot)[0].astype(np.int64)).to(cuda_device)
    G = [x.to(cuda_device) for x in (b.G1, b.G2, b.W, b.S2, b.n)]
    ctx = api.Context(nside, 45.0, "schirmer", nside_bin=nside)
    ctx.set_targets(tg)
    ctx.set_binned(*G)
    m1 = ctx.map_pixel()
    back = ctx.get_binned()
    px = torch.stack([G[0], G[1], G[3], G[2]], dim=1).contiguous()
    ctx.set_binned_packed(px, G[4])
    m2 = ctx.map_pixel()
    ctx.sync(60)
    for k in ("map_e", "map_b", "var", "sum_w", "count", "members"):
        assert torch.equal(m1[k], m2[k]), k
    for k, x in zip(("G1", "G2", "W", "S2", "n"), G):
        assert torch.equal(back[k], x), k


@pytest.mark.parametrize("ra0,dec0,no,nb", [(75.0, 5.0, 256, 512), (20.0, 70.0, 256, 256)])
def test_jarvis_filter_maps(cuda_device, ra0, dec0, no, nb):
    """The Gaussian-type filter of Jarvis et al. (2004), scale theta_ap / 4,
    through the tabulated-filter path of both map kernels."""
    cat = catalog(int(ra0 + dec0) + 900, 60_000, ra0, dec0, 3.5, nhalo=5, w_range=(0.5, 1.5), clumped=True)
    tg = cap_targets(no, ra0, dec0, 3.0)
    ctx, bf, px, _ = _gal_run(cuda_device, cat, tg, no, nb, 24.0, "jarvis", xc=0.25)
    rbf, rpx = _oracle_maps(cat, tg, no, nb, 24.0, 3, xc=0.25)
    _check(bf, rbf, "brute")
    _check(px, rpx, "pixel")


def test_pixel_map_at_nside_8192(cuda_device):
    """The largest grid (12 x 8192^2 = 8.05e8 pixels, full-sky arrays of 16 GB):
    a cap straddling the polar / equatorial boundary (dec 41.8), so both pixel
    kernels run, Schirmer 2'."""
    nside = 8192
    npix = 12 * nside * nside
    c = oracle.radec2vec([123.0], [41.8])[0]
    src = oracle.query_disc(nside, c, math.radians(0.35))
    rng = np.random.default_rng(8192)
    G1, G2, W, S2 = (np.zeros(npix, np.float32) for _ in range(4))
    n_p = np.zeros(npix, np.int32)
    n = rng.poisson(6.0, src.size).astype(np.int32)
    w = n * rng.uniform(0.5, 1.5, src.size)
    G1[src] = w * rng.normal(0.0, 0.3, src.size)
    G2[src] = w * rng.normal(0.0, 0.3, src.size)
    W[src] = w
    S2[src] = w * 0.3
    n_p[src] = n
    tg = np.sort(oracle.query_disc(nside, c, math.radians(0.25)))
    ctx = api.Context(nside, 2.0, "schirmer", nside_bin=nside)
    ctx.set_targets(torch.from_numpy(tg).to(cuda_device))
    ctx.set_binned(*(torch.from_numpy(x).to(cuda_device) for x in (G1, G2, W, S2, n_p)))
    got = ctx.map_pixel()
    ctx.sync(120)
    gen = ctx.general_targets().numel()
    assert 0 < gen < tg.size
    ref = oracle.finalise(oracle.aperture_pixels_f32(oracle.pix2vec(nside, tg), nside, G1, G2, W, S2, n_p, 2,
                                                     2.0 * ARCMIN), 2.0 * ARCMIN)
    _check(got, ref, "nside 8192")


def test_guard_band_targets_finished_in_place(cuda_device):
    """Targets of the general kernel with guard-band pairs take slots that a
    follow-up kernel finishes; a target that finds no free slot finishes
    itself with the same code.  The aperture radius is set to the chord
    between pixels three apart on polar ring 20 of NSIDE 64, so every target
    on that ring has pairs inside the float32 guard band: with one slot, all
    but one of them take the in-place path, and the maps stay bit-identical."""
    nside, ring = 64, 20
    z = 1.0 - ring * ring / (3.0 * nside * nside)
    rho = math.sqrt((1.0 - z) * (1.0 + z))
    theta_arcmin = 2.0 * math.asin(rho * math.sin(3 * (2 * math.pi / (4 * ring)) / 2)) / ARCMIN
    dec_ring = math.degrees(math.asin(z))
    cat = catalog(21, 60_000, 30.0, dec_ring, 8.0)
    tg = cap_targets(nside, 30.0, dec_ring, 5.0)
    on_ring = [p for p in tg if oracle.pix_info(nside, int(p))[0] == ring]
    assert len(on_ring) >= 4
    dev = cuda_device
    ctx = api.Context(nside, theta_arcmin, "schirmer", nside_bin=nside)
    c = cat.to(dev)
    ctx.set_targets(torch.from_numpy(tg).to(dev))
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    a = ctx.map_pixel()
    ctx.sync(60)
    n_fp64 = ctx.fp64_decisions()
    assert n_fp64 >= 2 * len(on_ring)
    ctx.set_band_slot_limit(1)
    b = ctx.map_pixel()
    ctx.sync(60)
    assert ctx.fp64_decisions() == n_fp64
    for k in ("map_e", "map_b", "var", "sum_w", "count", "members"):
        assert torch.equal(a[k], b[k]), k
    ctx.set_band_slot_limit(0)
    _, rpx = _oracle_maps(cat, tg, nside, nside, theta_arcmin, 2)
    _check(a, rpx, "guard band")


def _runs_of(pix):
    """Maximal runs of consecutive RING pixels: (first, length, offset)."""
    pix = np.asarray(pix, np.int64)
    brk = np.nonzero(np.diff(pix) != 1)[0] + 1
    starts = np.concatenate([[0], brk])
    ends = np.concatenate([brk, [pix.size]])
    return np.stack([pix[starts], ends - starts, starts], 1).astype(np.int64)


def test_binned_runs_equal_the_full_map(cuda_device):
    """A footprint given as runs of RING pixels (the cap crosses the azimuth
    seam, so rings split into two runs) gives the full-sky input's maps bit
    for bit; a second call with fewer runs and no clearing keeps the rest; a
    run outside the map is reported by the next sync."""
    nside = 256
    b, foot = binned_field_oracle(31, nside, 359.0, 20.0, 9.0, mean_count=12.0)
    tg = torch.from_numpy(np.nonzero(foot)[0].astype(np.int64)).to(cuda_device)
    full = [x.to(cuda_device) for x in (b.G1, b.G2, b.W, b.S2, b.n)]
    ctx = api.Context(nside, 25.0, "schirmer", nside_bin=nside)
    ctx.set_targets(tg)
    ctx.set_binned(*full)
    ref = {k: v.clone() for k, v in ctx.map_pixel().items()}
    pix = np.nonzero(foot)[0]
    runs = _runs_of(pix)
    assert (runs[:, 1] < 4 * nside).sum() > 0 and len(runs) > 40
    it = torch.from_numpy(pix).to(cuda_device)
    px = torch.stack([full[0], full[1], full[3], full[2]], 1)[it].contiguous()
    n_p = full[4][it].contiguous()
    rt = torch.from_numpy(runs).to(cuda_device)
    ctx.set_binned_runs(px, n_p, rt)
    got = ctx.map_pixel()
    ctx.sync(60)
    for k in ref:
        assert torch.equal(got[k], ref[k]), k
    # fewer runs, no clearing: the pixels of the other runs are kept
    ctx.set_binned_runs(px, n_p, rt[: len(runs) // 2])
    got = ctx.map_pixel()
    ctx.sync(60)
    for k in ref:
        assert torch.equal(got[k], ref[k]), k
    # clearing keeps only the given runs
    ctx.set_binned_runs(px, n_p, rt[: len(runs) // 2], clear=True)
    got = ctx.map_pixel()
    ctx.sync(60)
    assert not torch.equal(got["map_e"], ref["map_e"])
    # a run past the end of the map is skipped and reported
    bad = rt[:1].clone()
    bad[0, 0] = 12 * nside * nside
    ctx.set_binned_runs(px, n_p, bad)
    with pytest.raises(api.SmartError, match="SMART_E_ARG"):
        ctx.sync(60)
    ctx.close()
