"""FP64 CPU oracle for the spherical shear-based aperture mass (SMART).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2609_11181_b300``) and never imports it.

The heavy loops live in ``smart_oracle.c`` (plain C, binary64, compiled with
``-ffp-contract=off``); this module loads it with ctypes and adds numpy
wrappers.  Paper passages followed are cited per function (section /
equation of arXiv 2609.11181).  The MLP reference of the learned residual
correction lives in ``oracle/mlp.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smart_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FILTER_POLY = 1
FILTER_SCHIRMER = 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C source into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-std=c11", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i64, dbl, ip = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        L.orc_sincos_deg.argtypes = [dbl, ip, ip]
        L.orc_sincos_quarter.argtypes = [dbl, ip, ip]
        L.orc_pix_info.argtypes = [i64, i64, ip, ip, ip, ip, ip, ip]
        L.orc_pix2vec.argtypes = [i64, i64, ip]
        L.orc_ring_info.argtypes = [i64, i64, ip, ip, ip, ip]
        L.orc_ang2pix.argtypes = [i64, dbl, dbl]
        L.orc_ang2pix.restype = i64
        L.orc_ang2pix_many.argtypes = [i64, i64, ip, ip, ip]
        L.orc_pix2vec_many.argtypes = [i64, i64, ip, ip]
        L.orc_radec2vec.argtypes = [dbl, dbl, ip]
        L.orc_filter_q.argtypes = [ctypes.c_int, dbl, dbl]
        L.orc_filter_q.restype = dbl
        L.orc_filter_u_poly.argtypes = [dbl]
        L.orc_filter_u_poly.restype = dbl
        L.orc_aperture_galaxies.argtypes = [i64, ip, i64, ip, ip, ip, ip, ip,
                                            ctypes.c_int, dbl, dbl,
                                            ip, ip, ip, ip, ip]
        L.orc_query_disc.argtypes = [i64, ip, dbl, ip, i64]
        L.orc_query_disc.restype = i64
        L.orc_query_disc_all.argtypes = [i64, ip, dbl, ip, i64]
        L.orc_query_disc_all.restype = i64
        L.orc_aperture_pixels.argtypes = [i64, ip, i64, ip, ip, ip, ip, ip,
                                          ctypes.c_int, dbl, dbl,
                                          ip, ip, ip, ip, ip, ip]
        L.orc_aperture_pixels_f32.argtypes = L.orc_aperture_pixels.argtypes
        L.orc_finalise.argtypes = [i64, dbl, ip, ip, ip, ip, ip, ip, ip]
        L.orc_bin_catalog.argtypes = [i64, i64, ip, ip, ip, ip, ip,
                                      ip, ip, ip, ip, ip, ip, ip, ip]
        L.orc_barycentres.argtypes = [i64, ip, ip, ip, ip, ip, ip]
        L.orc_aperture_points.argtypes = [i64, ip, i64, ip, ip, ip, ip, ip, ip,
                                          ctypes.c_int, dbl, dbl,
                                          ip, ip, ip, ip, ip, ip]
        L.orc_project.argtypes = [dbl, dbl, i64, ip, ip, ip]
        L.orc_plane_shear.argtypes = [dbl, dbl, i64, ip, ip, ip, ip, ip]
        L.orc_aperture_projected.argtypes = [i64, ip, i64, ip, ip, ip, ip, ip, dbl, dbl,
                                             ctypes.c_int, dbl, dbl, ip, ip, ip, ip, ip]
        L.orc_finalise_area.argtypes = [i64, dbl, ip, ip, ip, ip, ip, ip, ip]
        L.orc_annulus_stats.argtypes = [i64, ip, ip, dbl, ip, ip, i64, ip, ip, ip]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


# --------------------------------------------------------------------------
# elementary functions and HEALPix (Sect. 3; Gorski et al. 2005)
# --------------------------------------------------------------------------
def sincos_deg(x: float):
    s, c = ctypes.c_double(), ctypes.c_double()
    lib().orc_sincos_deg(float(x), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def sincos_quarter(f: float):
    s, c = ctypes.c_double(), ctypes.c_double()
    lib().orc_sincos_quarter(float(f), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def pix_info(nside: int, pix: int):
    """(ring, j, nring, z, rho, phi_quarter_turns) of a RING pixel."""
    r, j, nr = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    z, rho, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_pix_info(nside, int(pix), ctypes.byref(r), ctypes.byref(j), ctypes.byref(nr),
                       ctypes.byref(z), ctypes.byref(rho), ctypes.byref(f))
    return r.value, j.value, nr.value, z.value, rho.value, f.value


def ring_info(nside: int, ring: int):
    """(first pixel, pixel count, z, shifted) of ring ``ring`` (1-based)."""
    s, n = ctypes.c_int64(), ctypes.c_int64()
    z, sh = ctypes.c_double(), ctypes.c_int()
    lib().orc_ring_info(nside, int(ring), ctypes.byref(s), ctypes.byref(n),
                        ctypes.byref(z), ctypes.byref(sh))
    return s.value, n.value, z.value, bool(sh.value)


def ang2pix(nside: int, ra_deg, dec_deg) -> np.ndarray:
    ra, dec = _f64(ra_deg).ravel(), _f64(dec_deg).ravel()
    out = np.empty(ra.size, dtype=np.int64)
    lib().orc_ang2pix_many(nside, ra.size, _p(ra), _p(dec), _p(out))
    return out


def pix2vec(nside: int, pix) -> np.ndarray:
    p = _i64(pix).ravel()
    out = np.empty((p.size, 3), dtype=np.float64)
    lib().orc_pix2vec_many(nside, p.size, _p(p), _p(out))
    return out


def radec2vec(ra_deg, dec_deg) -> np.ndarray:
    ra, dec = _f64(ra_deg).ravel(), _f64(dec_deg).ravel()
    out = np.empty((ra.size, 3), dtype=np.float64)
    v = np.empty(3)
    for k in range(ra.size):
        lib().orc_radec2vec(ra[k], dec[k], _p(v))
        out[k] = v
    return out


def chord2(theta_ap: float) -> float:
    """T = 4 sin^2(theta_ap / 2): a point is in the aperture iff s^2 <= T."""
    return 4.0 * np.sin(0.5 * theta_ap) ** 2


def query_disc(nside: int, r0, theta_ap: float, all_pixels: bool = False) -> np.ndarray:
    """RING pixels whose centres lie within theta_ap of r0 (Sect. 3.2, ring intervals)."""
    v = _f64(r0)
    T = chord2(theta_ap)
    cap = int(2 * 2 * np.pi * (1 - np.cos(theta_ap)) / (4 * np.pi / (12 * nside * nside))) + 16 * nside + 64
    buf = np.empty(cap, dtype=np.int64)
    fn = lib().orc_query_disc_all if all_pixels else lib().orc_query_disc
    m = fn(nside, _p(v), T, _p(buf), cap)
    return buf[:min(m, cap)].copy()


# --------------------------------------------------------------------------
# filters (Sect. 2, Eq. 5; Schneider 1996; Schirmer et al. 2007)
# --------------------------------------------------------------------------
def filter_q(kind: int, x, xc: float = 0.15) -> np.ndarray:
    xs = np.atleast_1d(_f64(x))
    return np.array([lib().orc_filter_q(kind, xc, float(v)) for v in xs])


def filter_u_poly(x) -> np.ndarray:
    xs = np.atleast_1d(_f64(x))
    return np.array([lib().orc_filter_u_poly(float(v)) for v in xs])


# --------------------------------------------------------------------------
# aperture sums (Sect. 3.1 brute force, Sect. 3.2 pixel-based) and the
# summed normalisation (Sect. 2.4)
# --------------------------------------------------------------------------
def aperture_galaxies(centres, ra, dec, e1, e2, w, kind, theta_ap, xc=0.15):
    """Brute-force sums at unit-vector centres over a galaxy catalogue.

    Returns dict(SE, SB, SV, SW, N).  Sect. 3.1 steps 1-4 (sphS_pos).
    """
    c = _f64(centres).reshape(-1, 3)
    ra, dec, e1, e2, w = (_f64(a).ravel() for a in (ra, dec, e1, e2, w))
    n0, n = c.shape[0], ra.size
    SE, SB, SV, SW = (np.empty(n0) for _ in range(4))
    N = np.empty(n0, dtype=np.int64)
    lib().orc_aperture_galaxies(n0, _p(c), n, _p(ra), _p(dec), _p(e1), _p(e2), _p(w),
                                int(kind), float(xc), float(theta_ap),
                                _p(SE), _p(SB), _p(SV), _p(SW), _p(N))
    return dict(SE=SE, SB=SB, SV=SV, SW=SW, N=N)


def aperture_pixels(centres, nside_bin, G1, G2, W, S2, n_p, kind, theta_ap, xc=0.15):
    """Pixel-based sums at unit-vector centres over a full-sky binned map.

    Returns dict(SE, SB, SV, SW, N, NPIX).  Sect. 3.2 steps 3-5 (sphS_pix).
    """
    c = _f64(centres).reshape(-1, 3)
    G1, G2, W, S2 = (_f64(a).ravel() for a in (G1, G2, W, S2))
    n_p = _i64(n_p).ravel()
    assert G1.size == 12 * nside_bin * nside_bin
    n0 = c.shape[0]
    SE, SB, SV, SW = (np.empty(n0) for _ in range(4))
    N = np.empty(n0, dtype=np.int64)
    NP = np.empty(n0, dtype=np.int64)
    lib().orc_aperture_pixels(n0, _p(c), nside_bin, _p(G1), _p(G2), _p(W), _p(S2), _p(n_p),
                              int(kind), float(xc), float(theta_ap),
                              _p(SE), _p(SB), _p(SV), _p(SW), _p(N), _p(NP))
    return dict(SE=SE, SB=SB, SV=SV, SW=SW, N=N, NPIX=NP)


def aperture_pixels_f32(centres, nside_bin, G1, G2, W, S2, n_p, kind, theta_ap, xc=0.15):
    """As aperture_pixels, reading float32 sums / int32 counts without a copy."""
    c = _f64(centres).reshape(-1, 3)
    G1, G2, W, S2 = (np.ascontiguousarray(a, dtype=np.float32).ravel() for a in (G1, G2, W, S2))
    n_p = np.ascontiguousarray(n_p, dtype=np.int32).ravel()
    assert G1.size == 12 * nside_bin * nside_bin
    n0 = c.shape[0]
    SE, SB, SV, SW = (np.empty(n0) for _ in range(4))
    N = np.empty(n0, dtype=np.int64)
    NP = np.empty(n0, dtype=np.int64)
    lib().orc_aperture_pixels_f32(n0, _p(c), nside_bin, _p(G1), _p(G2), _p(W), _p(S2), _p(n_p),
                                  int(kind), float(xc), float(theta_ap),
                                  _p(SE), _p(SB), _p(SV), _p(SW), _p(N), _p(NP))
    return dict(SE=SE, SB=SB, SV=SV, SW=SW, N=N, NPIX=NP)


def finalise(sums: dict, theta_ap: float) -> dict:
    """Summed normalisation, Sect. 2.4 / Sect. 3.1 step 5, Eq. 8."""
    SE, SB, SV, SW = (_f64(sums[k]) for k in ("SE", "SB", "SV", "SW"))
    n0 = SE.size
    ME, MB, VAR = (np.empty(n0) for _ in range(3))
    lib().orc_finalise(n0, float(theta_ap), _p(SE), _p(SB), _p(SV), _p(SW), _p(ME), _p(MB), _p(VAR))
    out = dict(sums)
    out.update(ME=ME, MB=MB, VAR=VAR)
    return out


def map_galaxies(centres, ra, dec, e1, e2, w, kind, theta_ap, xc=0.15):
    return finalise(aperture_galaxies(centres, ra, dec, e1, e2, w, kind, theta_ap, xc), theta_ap)


def map_pixels(centres, nside_bin, G1, G2, W, S2, n_p, kind, theta_ap, xc=0.15):
    return finalise(aperture_pixels(centres, nside_bin, G1, G2, W, S2, n_p, kind, theta_ap, xc),
                    theta_ap)


def bin_catalog(nside: int, ra, dec, e1, e2, w) -> dict:
    """Stable sort by RING pixel + offsets + per-pixel sums (Sect. 3.4, Sect. 3.2 step 2)."""
    ra, dec, e1, e2, w = (_f64(a).ravel() for a in (ra, dec, e1, e2, w))
    n = ra.size
    npix = 12 * nside * nside
    pix = np.empty(n, dtype=np.int64)
    perm = np.empty(n, dtype=np.int64)
    offsets = np.empty(npix + 1, dtype=np.int64)
    G1, G2, W, S2 = (np.empty(npix) for _ in range(4))
    n_p = np.empty(npix, dtype=np.int64)
    lib().orc_bin_catalog(nside, n, _p(ra), _p(dec), _p(e1), _p(e2), _p(w),
                          _p(pix), _p(perm), _p(offsets), _p(G1), _p(G2), _p(W), _p(S2), _p(n_p))
    return dict(pix=pix, perm=perm, offsets=offsets, G1=G1, G2=G2, W=W, S2=S2, n=n_p)


def barycentres(nside: int, ra, dec, w, binned: dict) -> dict:
    """Pixels holding galaxies and their w-weighted mean unit vectors (Sect. 3.3),
    summed in the order of bin_catalog's permutation."""
    ra, dec, w = (_f64(a).ravel() for a in (ra, dec, w))
    npix = 12 * nside * nside
    vec = np.zeros((npix, 3))
    lib().orc_barycentres(nside, _p(ra), _p(dec), _p(w), _p(_i64(binned["perm"])), _p(_i64(binned["offsets"])),
                          _p(vec))
    pix = np.nonzero(binned["n"] > 0)[0]
    return dict(pix=pix, vec=np.ascontiguousarray(vec[pix]))


def aperture_points(centres, vec, G1, G2, W, S2, n_p, kind, theta_ap, xc=0.15):
    """Sums at unit-vector centres over weighted points (barycentre form, Sect. 3.3)."""
    c = _f64(centres).reshape(-1, 3)
    v = _f64(vec).reshape(-1, 3)
    G1, G2, W, S2 = (_f64(a).ravel() for a in (G1, G2, W, S2))
    n_p = _i64(n_p).ravel()
    n0, m = c.shape[0], v.shape[0]
    SE, SB, SV, SW = (np.empty(n0) for _ in range(4))
    N = np.empty(n0, dtype=np.int64)
    K = np.empty(n0, dtype=np.int64)
    lib().orc_aperture_points(n0, _p(c), m, _p(v), _p(G1), _p(G2), _p(W), _p(S2), _p(n_p), int(kind), float(xc),
                              float(theta_ap), _p(SE), _p(SB), _p(SV), _p(SW), _p(N), _p(K))
    return dict(SE=SE, SB=SB, SV=SV, SW=SW, N=N, K=K)


def map_barycentre(centres, nside_bin, ra, dec, e1, e2, w, kind, theta_ap, xc=0.15):
    """The barycentre form of the pixel-based map (Sect. 3.3, sphS_pixB), summed normalisation."""
    b = bin_catalog(nside_bin, ra, dec, e1, e2, w)
    bc = barycentres(nside_bin, ra, dec, w, b)
    p = bc["pix"]
    return finalise(aperture_points(centres, bc["vec"], b["G1"][p], b["G2"][p], b["W"][p], b["S2"][p], b["n"][p],
                                    kind, theta_ap, xc), theta_ap)


# --------------------------------------------------------------------------
# averaged normalisation (Sect. 2.4): each bin pixel's shear is normalised by
# its own weight and multiplied by the pixel area (the analogue of the
# convergence-based map, Sect. 5.3 step 2); no aperture density.
#   M_E = sum_p Q (G+_p / W_p) A_pix,  sigma^2 = 1/2 sum_p Q^2 S2_p (A_pix / W_p)^2
# For galaxies each one carries w A_pix / W of its bin pixel.
# --------------------------------------------------------------------------
def _averaged(sums: dict) -> dict:
    out = dict(sums)
    out.update(ME=np.asarray(sums["SE"], np.float64), MB=np.asarray(sums["SB"], np.float64),
               VAR=0.5 * np.asarray(sums["SV"], np.float64))
    return out


def _avg_scale(nside_bin: int, W) -> np.ndarray:
    W = np.asarray(W, np.float64)
    apix = 4.0 * np.pi / (12.0 * nside_bin * nside_bin)
    return np.divide(apix, W, out=np.zeros_like(W), where=W > 0)


def map_pixels_averaged(centres, nside_bin, G1, G2, W, S2, n_p, kind, theta_ap, xc=0.15):
    f = _avg_scale(nside_bin, W)
    G1, G2, S2 = (np.asarray(a, np.float64) for a in (G1, G2, S2))
    return _averaged(aperture_pixels(centres, nside_bin, G1 * f, G2 * f, W, S2 * f * f, n_p, kind, theta_ap, xc))


def map_galaxies_averaged(centres, nside_bin, ra, dec, e1, e2, w, kind, theta_ap, xc=0.15):
    b = bin_catalog(nside_bin, ra, dec, e1, e2, w)
    f = _avg_scale(nside_bin, b["W"])[b["pix"]]
    return _averaged(aperture_galaxies(centres, ra, dec, e1, e2, np.asarray(w, np.float64) * f, kind, theta_ap, xc))


def map_barycentre_averaged(centres, nside_bin, ra, dec, e1, e2, w, kind, theta_ap, xc=0.15):
    b = bin_catalog(nside_bin, ra, dec, e1, e2, w)
    bc = barycentres(nside_bin, ra, dec, w, b)
    p = bc["pix"]
    f = _avg_scale(nside_bin, b["W"][p])
    return _averaged(aperture_points(centres, bc["vec"], b["G1"][p] * f, b["G2"][p] * f, b["W"][p],
                                     b["S2"][p] * f * f, b["n"][p], kind, theta_ap, xc))


# --------------------------------------------------------------------------
# Cartesian (projected) estimator, projS_pos (Sect. 2.2, Sect. 5.2.1), and the
# equal-area annulus statistics of Sect. 5.2.2
# --------------------------------------------------------------------------
def project(ra_c: float, dec_c: float, vec):
    """Gnomonic plane coordinates (n, 2) about (ra_c, dec_c) of unit vectors
    (n, 3), and a flag per point (False: no image, r . c <= 0)."""
    v = _f64(vec).reshape(-1, 3)
    xy = np.empty((v.shape[0], 2))
    ok = np.empty(v.shape[0], dtype=np.int64)
    lib().orc_project(float(ra_c), float(dec_c), v.shape[0], _p(v), _p(xy), _p(ok))
    return xy, ok.astype(bool)


def plane_shear(ra_c: float, dec_c: float, ra, dec, e1, e2) -> np.ndarray:
    """Shear components (n, 2) in the plane's axes, rotated with the local
    North (Sect. 2.2.2)."""
    ra, dec, e1, e2 = (_f64(a).ravel() for a in (ra, dec, e1, e2))
    g = np.empty((ra.size, 2))
    lib().orc_plane_shear(float(ra_c), float(dec_c), ra.size, _p(ra), _p(dec), _p(e1), _p(e2), _p(g))
    return g


def aperture_projected(centres, ra, dec, e1, e2, w, ra_c, dec_c, kind, theta_ap, xc=0.15):
    """Cartesian brute-force sums at unit-vector centres (projS_pos)."""
    c = _f64(centres).reshape(-1, 3)
    ra, dec, e1, e2, w = (_f64(a).ravel() for a in (ra, dec, e1, e2, w))
    n0, n = c.shape[0], ra.size
    SE, SB, SV, SW = (np.empty(n0) for _ in range(4))
    N = np.empty(n0, dtype=np.int64)
    lib().orc_aperture_projected(n0, _p(c), n, _p(ra), _p(dec), _p(e1), _p(e2), _p(w), float(ra_c), float(dec_c),
                                 int(kind), float(xc), float(theta_ap), _p(SE), _p(SB), _p(SV), _p(SW), _p(N))
    return dict(SE=SE, SB=SB, SV=SV, SW=SW, N=N)


def finalise_area(sums: dict, area: float) -> dict:
    """Summed normalisation with aperture area `area` (sr)."""
    SE, SB, SV, SW = (_f64(sums[k]) for k in ("SE", "SB", "SV", "SW"))
    n0 = SE.size
    ME, MB, VAR = (np.empty(n0) for _ in range(3))
    lib().orc_finalise_area(n0, float(area), _p(SE), _p(SB), _p(SV), _p(SW), _p(ME), _p(MB), _p(VAR))
    out = dict(sums)
    out.update(ME=ME, MB=MB, VAR=VAR)
    return out


def map_projected(centres, ra, dec, e1, e2, w, ra_c, dec_c, kind, theta_ap, xc=0.15):
    """projS_pos map (Sect. 5.2.1): plane sums normalised with A = pi theta_ap^2."""
    return finalise_area(aperture_projected(centres, ra, dec, e1, e2, w, ra_c, dec_c, kind, theta_ap, xc),
                         np.pi * theta_ap * theta_ap)


def annulus_stats(centres, ref_vec, rmax: float, m_x, m_ref, nbins: int):
    """Equal-area annuli about ref_vec out to rmax (rad): count, mean and
    population sd of (m_x - m_ref) / sd(m_ref) per annulus (Sect. 5.2.2)."""
    c = _f64(centres).reshape(-1, 3)
    r = _f64(ref_vec).ravel()
    mx, mr = _f64(m_x).ravel(), _f64(m_ref).ravel()
    cnt = np.empty(nbins, dtype=np.int64)
    mean, sd = np.empty(nbins), np.empty(nbins)
    lib().orc_annulus_stats(c.shape[0], _p(c), _p(r), float(rmax), _p(mx), _p(mr), int(nbins), _p(cnt), _p(mean),
                            _p(sd))
    return dict(count=cnt, mean=mean, sd=sd)


def rms_rel(a, b) -> float:
    """rms(a - b) / rms(b): the map parity statistic."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    den = np.sqrt(np.mean(b * b))
    return float(np.sqrt(np.mean((a - b) ** 2)) / den) if den > 0 else float(np.sqrt(np.mean(a * a)))


def epsilon_stats(m_x, m_ref):
    """Sect. 5.1, Eq. 12: eps_X = (M_X - M_ref) / sigma(M_ref); returns (mean, std)."""
    m_x, m_ref = np.asarray(m_x, np.float64), np.asarray(m_ref, np.float64)
    eps = (m_x - m_ref) / np.std(m_ref)
    return float(np.mean(eps)), float(np.std(eps))
