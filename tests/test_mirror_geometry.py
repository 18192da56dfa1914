"""The HEALPix symmetry the general kernel's mirror pairs rest on, checked
against the oracle's pixel centres (no GPU): on every ring of nr = 4 q
pixels centred at azimuths (j + s/2) 2 pi / nr, the pixel at azimuth phi has
its mirror image about the meridian m pi/4 (m = 0..3) at index
(m q - s - j) mod nr, on the same ring (the HEALPix ring scheme of Gorski
et al. 2005)."""
import math

import numpy as np
import pytest

import oracle


def _rings(nside):
    start = 0
    for ring in range(1, 4 * nside):
        if ring < nside:
            nr, s = 4 * ring, 1
        elif ring <= 3 * nside:
            nr, s = 4 * nside, 1 if (ring - nside) % 2 == 0 else 0
        else:
            nr, s = 4 * (4 * nside - ring), 1
        yield start, nr, s
        start += nr


@pytest.mark.parametrize("nside", [1, 2, 4, 16, 64])
def test_mirror_index_maps_centres_to_their_images(nside):
    n = 0
    for start, nr, s in _rings(nside):
        j = np.arange(nr)
        v = oracle.pix2vec(nside, start + j)
        phi = np.arctan2(v[:, 1], v[:, 0])
        q = nr // 4
        for m in range(4):
            jm = (m * q - s - j) % nr
            # same ring (same z), azimuth m pi/2 - phi
            assert np.array_equal(v[jm, 2], v[:, 2])
            d = (phi[jm] - (m * math.pi / 2 - phi) + math.pi) % (2 * math.pi) - math.pi
            assert np.abs(d).max() < 1e-12
            # an involution
            assert np.array_equal((m * q - s - jm) % nr, j)
        n += nr
    assert n == 12 * nside * nside


def test_mirror_pairs_share_the_pair_geometry():
    """For a target and its image, every pair (image, image of bin pixel k)
    has the chord of the pair (target, k), and the tangent-plane direction
    mirrored (x -> -x, y unchanged), so cos 2psi is shared and sin 2psi
    changes sign: checked from unit vectors at NSIDE 32 on rings of both
    kinds, for bin rings above and below the target's."""
    nside = 32
    rings = list(_rings(nside))
    rng = np.random.default_rng(3)
    for ring in (5, 20, 31, 40, 64, 100):
        start, nr, s = rings[ring - 1]
        for _ in range(4):
            j = int(rng.integers(nr))
            m = int(rng.integers(4))
            jm = (m * (nr // 4) - s - j) % nr
            t, ti = oracle.pix2vec(nside, [start + j, start + jm])
            for dr in (-3, 0, 2):
                bstart, bnr, bs = rings[ring - 1 + dr]
                k = np.arange(bnr)
                km = (m * (bnr // 4) - bs - k) % bnr
                p = oracle.pix2vec(nside, bstart + k)
                pi_ = oracle.pix2vec(nside, bstart + km)
                c1 = ((p - t) ** 2).sum(1)
                c2 = ((pi_ - ti) ** 2).sum(1)
                assert np.abs(c1 - c2).max() < 1e-13
                # direction of the target in the pixel's (East, North) basis
                def en(pt, tg):
                    e = np.stack([-pt[:, 1], pt[:, 0], np.zeros(len(pt))], 1)
                    e /= np.linalg.norm(e, axis=1)[:, None]
                    nn = np.cross(pt, e)
                    d = tg - pt
                    return (d * e).sum(1), (d * nn).sum(1)
                x1, y1 = en(p, t)
                x2, y2 = en(pi_, ti)
                assert np.abs(x1 + x2).max() < 1e-12 and np.abs(y1 - y2).max() < 1e-12
