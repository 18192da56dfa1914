"""The catalogue sort that allocates no device memory.

``smart_sort_catalog_noalloc`` serves callers that cannot allocate device
memory when they need the sort: code confined to a fixed memory budget from
its own pool, host threads that must not take the device-wide
synchronisation of cudaMalloc/cudaFree, and runtimes that forbid allocation
inside their scheduling regions.  Its working memory is one fixed array in
the library's device data, shared by every call.

The GPU test runs it twice in a row on different catalogues (the second
smaller and at another NSIDE, so anything the first call left in the shared
array would show) and requires the result of each call to equal, bit for
bit, the sort of the context path (smart_bin_galaxies + smart_get_catalog).
A second test sorts points placed on the pixel boundaries and compares the
keys with the oracle's ang2pix.  The file is named so that pytest collects it last; it passes alone in a
fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2609_11181_b300 import _native as N
from paper_2609_11181_b300 import api

from _cases import boundary_points, catalog

MAX_GALAXIES = 1 << 20
SMART_E_ARG, SMART_E_OVERFLOW = 1, 6


def _noalloc_sort(lib, nside, ra, dec, stream):
    n = ra.numel()
    dev = ra.device
    pix = torch.empty(n, dtype=torch.int32, device=dev)        # uint32 in the C ABI
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    off = torch.empty(12 * nside * nside + 1, dtype=torch.int32, device=dev)
    st = lib.smart_sort_catalog_noalloc(nside, ra.data_ptr(), dec.data_ptr(), n, pix.data_ptr(),
                                        perm.data_ptr(), off.data_ptr(), stream)
    assert st == 0, N.STATUS.get(st, st)
    return pix, perm, off


def _context_sort(nside, cat, dev):
    ctx = api.Context(nside, 10.0, "poly", nside_bin=nside)
    c = cat.to(dev)
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    perm, pix, off = ctx.get_catalog(c.ra_deg.numel())
    ctx.sync(60)
    out = (pix.clone(), perm.clone(), off.clone())
    ctx.close()
    return out


@pytest.mark.gpu
def test_noalloc_sort_matches_context_sort_twice(cuda_device):
    lib = N.load()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        # (nside, catalogue): the first at the size limit with an odd number of
        # radix passes (24-bit keys, three passes), the second smaller with
        # four passes
        (1024, catalog(71, MAX_GALAXIES, 30.0, 10.0, 8.0, nhalo=4, clumped=True)),
        (2048, catalog(72, 200_001, 210.0, -50.0, 3.0, nhalo=3)),
    ]
    for nside, cat in cases:
        ra, dec = cat.ra_deg.to(cuda_device), cat.dec_deg.to(cuda_device)
        pix, perm, off = _noalloc_sort(lib, nside, ra, dec, stream)
        torch.cuda.synchronize()
        ref_pix, ref_perm, ref_off = _context_sort(nside, cat, cuda_device)
        assert torch.equal(pix.long(), ref_pix), f"nside {nside}: pixel keys differ"
        assert torch.equal(perm.long(), ref_perm), f"nside {nside}: permutation differs"
        assert torch.equal(off.long(), ref_off), f"nside {nside}: offsets differ"
        assert int(off[-1]) == ra.numel()


@pytest.mark.gpu
@pytest.mark.parametrize("nside", [256, 8192])
def test_noalloc_keys_at_pixel_boundaries(cuda_device, nside):
    # this entry point computes every key with the float64 definition, the
    # context path with float32 where that is certain: on points placed at
    # every kind of pixel boundary both equal the oracle's ang2pix
    lib = N.load()
    stream = torch.cuda.current_stream().cuda_stream
    ra, dec = boundary_points(nside, 40_000, nside + 1)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda_device, torch.float64)
    pix, perm, off = _noalloc_sort(lib, nside, t(ra), t(dec), stream)
    torch.cuda.synchronize()
    ref = oracle.ang2pix(nside, ra, dec)
    ref_perm = np.argsort(ref, kind="stable")
    np.testing.assert_array_equal(pix.cpu().numpy().astype(np.int64), ref[ref_perm])
    np.testing.assert_array_equal(perm.cpu().numpy().astype(np.int64), ref_perm)
    np.testing.assert_array_equal(off.cpu().numpy()[ref[ref_perm]], np.searchsorted(ref[ref_perm], ref[ref_perm]))


def test_noalloc_sort_rejects_bad_sizes():
    # checked on the host before any device work, so no GPU is needed
    lib = N.load()
    dummy = ctypes.c_void_p(16)
    assert lib.smart_sort_catalog_noalloc(3, dummy, dummy, 10, dummy, dummy, dummy, None) == SMART_E_ARG
    assert lib.smart_sort_catalog_noalloc(16384, dummy, dummy, 10, dummy, dummy, dummy, None) == SMART_E_ARG
    assert lib.smart_sort_catalog_noalloc(64, dummy, dummy, -1, dummy, dummy, dummy, None) == SMART_E_ARG
    assert lib.smart_sort_catalog_noalloc(64, None, dummy, 10, dummy, dummy, dummy, None) == SMART_E_ARG
    assert (lib.smart_sort_catalog_noalloc(64, dummy, dummy, MAX_GALAXIES + 1, dummy, dummy, dummy, None)
            == SMART_E_OVERFLOW)
