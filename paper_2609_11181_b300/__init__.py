"""B300-native spherical shear-based aperture-mass maps (SMART, arXiv 2609.11181).

The compute path is the CUDA library ``_lib/libsmart.so`` (sources in
``csrc/``, C ABI in ``include/smart.h``); ``api`` is a thin ctypes binding.
``synth`` makes the seeded synthetic inputs.
"""
__all__ = ["api", "synth", "build"]
