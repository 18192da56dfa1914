"""CPU-side checks of the CUDA library: it loads without a GPU, exports every
symbol that include/smart.h declares, and rejects bad arguments on the host
before any device work.  No compute call is made here."""
import ctypes
import math
import os
import re

import pytest

import oracle
from paper_2609_11181_b300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(smart_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = N.load()
    decl = _declared()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(lib, name), name
    assert decl == set(N.SIGNATURES), decl ^ set(N.SIGNATURES)


@pytest.mark.parametrize("arcmin", [0.5, 10.0, 15.0, 60.0, 600.0])
def test_chord_threshold_matches_oracle(arcmin):
    # both sides must use the identical float64 threshold T
    th = arcmin * math.pi / 10800
    T = N.load().smart_chord2(arcmin)
    assert T == 4.0 * math.sin(0.5 * th) ** 2
    assert T == oracle.chord2(th)


def test_create_rejects_bad_arguments():
    lib = N.load()
    h = ctypes.c_void_p()
    f = N.SmartFilter(N.FILTER_POLY, 0.15)
    bad = [(3, 10.0, 64), (64, 0.0, 64), (64, -1.0, 64), (64, 10.0, 16384), (0, 10.0, 64),
           (64, float("nan"), 64), (64, 1e9, 64)]
    for nside, th, nb in bad:
        assert lib.smart_create(nside, ctypes.byref(f), th, nb, None, ctypes.byref(h)) == 1
        assert h.value is None
    f2 = N.SmartFilter(7, 0.15)
    assert lib.smart_create(64, ctypes.byref(f2), 10.0, 64, None, ctypes.byref(h)) == 1
    f3 = N.SmartFilter(N.FILTER_SCHIRMER, -0.1)
    assert lib.smart_create(64, ctypes.byref(f3), 10.0, 64, None, ctypes.byref(h)) == 1
    assert lib.smart_create(64, None, 10.0, 64, None, ctypes.byref(h)) == 1


def test_stateless_calls_reject_bad_arguments():
    lib = N.load()
    assert lib.smart_ang2pix(3, None, None, 10, None, None) == 1
    assert lib.smart_ang2pix(64, None, None, -1, None, None) == 1
    assert lib.smart_ang2pix(64, None, None, 5, None, None) == 1
    assert lib.smart_ang2pix(64, None, None, 0, None, None) == 0      # empty input is fine
    assert lib.smart_pix2vec(64, None, 3, None, None) == 1
    assert lib.smart_sync(None, 1.0) == 1
    assert lib.smart_set_band_slot_limit(None, 1) == 1
    n1, n2 = ctypes.c_int64(), ctypes.c_int64()
    assert lib.smart_get_general_pairs(None, None, 0, ctypes.byref(n1), ctypes.byref(n2)) == 1
    assert lib.smart_last_error(None) == b"null context"
    lib.smart_destroy(None)
    fl = ctypes.c_double(0.0)
    for bits in (16, 33, 64 | 0x100, 0x100):            # packed form is float32 only
        assert lib.smart_fma_probe(bits, 4, 1, None, ctypes.byref(fl)) == 1
    assert lib.smart_fma_probe(32, 0, 1, None, ctypes.byref(fl)) == 1
    assert lib.smart_fma_probe(32, 4, 9, None, ctypes.byref(fl)) == 1
    assert lib.smart_fma_probe(32, 4, 1, None, None) == 1
