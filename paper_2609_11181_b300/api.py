"""Python binding of the SMART C ABI (argument marshalling only).

Every step of the computation runs in the CUDA library; this module checks
tensor devices/dtypes, passes raw device pointers and the current torch
stream, and turns status codes into exceptions.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _native as N
from ._native import SmartError

ARCMIN = math.pi / 10800.0


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor | None, dtype: torch.dtype, name: str, n: int | None = None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def chord2(theta_ap_arcmin: float) -> float:
    """T = 4 sin^2(theta_ap/2) as the library computes it (host helper)."""
    return N.load().smart_chord2(float(theta_ap_arcmin))


def ang2pix(nside: int, ra_deg: torch.Tensor, dec_deg: torch.Tensor) -> torch.Tensor:
    n = ra_deg.numel()
    out = torch.empty(n, dtype=torch.int64, device=ra_deg.device)
    st = N.load().smart_ang2pix(nside, _ptr(ra_deg, torch.float64, "ra"), _ptr(dec_deg, torch.float64, "dec", n),
                                n, _ptr(out, torch.int64, "pix"), _stream_handle())
    if st:
        raise SmartError(st, "smart_ang2pix")
    return out


def pix2vec(nside: int, pix: torch.Tensor) -> torch.Tensor:
    n = pix.numel()
    out = torch.empty((n, 3), dtype=torch.float64, device=pix.device)
    st = N.load().smart_pix2vec(nside, _ptr(pix, torch.int64, "pix"), n, _ptr(out, torch.float64, "vec"),
                                _stream_handle())
    if st:
        raise SmartError(st, "smart_pix2vec")
    return out


PROBE_PACKED = 0x100


def fma_probe(bits: int, iters: int, ctas_per_sm: int = 8, stream=None, packed: bool = False) -> float:
    """Enqueue the FMA throughput probe (float32 or float64; packed=True: float32
    pairs through the packed two-lane instruction) on the stream and return its
    floating-point operation count; time it with events."""
    flops = ctypes.c_double(0.0)
    st = N.load().smart_fma_probe(int(bits) | (PROBE_PACKED if packed else 0), int(iters), int(ctas_per_sm),
                                  _stream_handle(stream), ctypes.byref(flops))
    if st:
        raise SmartError(st, "smart_fma_probe")
    return flops.value


class Context:
    """One aperture-mass problem: output grid, filter, aperture, bin grid."""

    def __init__(self, nside_out: int, theta_ap_arcmin: float, filter: str = "poly", xc: float | None = None,
                 nside_bin: int | None = None, stream: torch.cuda.Stream | None = None):
        self._lib = N.load()
        kind = {"poly": N.FILTER_POLY, "schirmer": N.FILTER_SCHIRMER, "jarvis": N.FILTER_JARVIS}[filter]
        if xc is None:
            xc = 0.25 if filter == "jarvis" else 0.15
        f = N.SmartFilter(kind, float(xc))
        h = ctypes.c_void_p()
        self._stream = stream
        self.nside_out = int(nside_out)
        self.nside_bin = int(nside_bin if nside_bin is not None else nside_out)
        self.theta_ap_arcmin = float(theta_ap_arcmin)
        self.filter = filter
        self.xc = float(xc)
        st = self._lib.smart_create(self.nside_out, ctypes.byref(f), self.theta_ap_arcmin, self.nside_bin,
                                    _stream_handle(stream), ctypes.byref(h))
        if st:
            raise SmartError(st, "smart_create")
        self._h = h
        self._keep = []
        self.n_targets = 0

    # -- plumbing
    def _check(self, st: int, what: str):
        if st:
            msg = self._lib.smart_last_error(self._h)
            raise SmartError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.smart_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def npix_bin(self) -> int:
        return 12 * self.nside_bin * self.nside_bin

    # -- inputs
    def set_targets(self, pix: torch.Tensor):
        n = pix.numel()
        self._check(self._lib.smart_set_targets(self._h, _ptr(pix, torch.int64, "targets"), n), "smart_set_targets")
        self.n_targets = n

    def bin_galaxies(self, ra_deg, dec_deg, e1, e2, w=None):
        n = ra_deg.numel()
        self._check(self._lib.smart_bin_galaxies(
            self._h, _ptr(ra_deg, torch.float64, "ra", n), _ptr(dec_deg, torch.float64, "dec", n),
            _ptr(e1, torch.float32, "e1", n), _ptr(e2, torch.float32, "e2", n),
            _ptr(w, torch.float32, "w", n), n), "smart_bin_galaxies")

    def set_binned(self, G1, G2, W, S2, n_p):
        m = self.npix_bin
        self._check(self._lib.smart_set_binned(
            self._h, _ptr(G1, torch.float32, "G1", m), _ptr(G2, torch.float32, "G2", m),
            _ptr(W, torch.float32, "W", m), _ptr(S2, torch.float32, "S2", m), _ptr(n_p, torch.int32, "n_p", m)),
            "smart_set_binned")
        self._keep = [G1, G2, W, S2, n_p]

    def set_binned_packed(self, px, n_p):
        """px: float32 tensor of shape (npix, 4) holding (G1, G2, S2, W) per pixel; borrowed."""
        m = self.npix_bin
        if px.dim() != 2 or px.shape[1] != 4:
            raise ValueError("px must have shape (npix, 4)")
        self._check(self._lib.smart_set_binned_packed(
            self._h, _ptr(px, torch.float32, "px", 4 * m), _ptr(n_p, torch.int32, "n_p", m)),
            "smart_set_binned_packed")
        self._keep = [px, n_p]

    def set_binned_runs(self, px, n_p, runs, clear: bool = False):
        """Footprint input: px (m, 4) float32 and n_p (m,) int32 hold the pixels
        of the runs back to back; runs (k, 3) int64 = (first RING pixel,
        length, offset into px).  Copied into the context's own map."""
        m = n_p.numel()
        if px.dim() != 2 or px.shape[1] != 4 or px.shape[0] != m:
            raise ValueError("px must have shape (m, 4) with m = n_p.numel()")
        if runs.dim() != 2 or runs.shape[1] != 3:
            raise ValueError("runs must have shape (k, 3)")
        self._check(self._lib.smart_set_binned_runs(
            self._h, _ptr(px, torch.float32, "px"), _ptr(n_p, torch.int32, "n_p"), _ptr(runs, torch.int64, "runs"),
            runs.shape[0], m, 1 if clear else 0), "smart_set_binned_runs")
        self._keep = [px, n_p, runs]

    # -- maps
    def _out(self, out):
        if out is None:
            dev = torch.device("cuda", torch.cuda.current_device())
            n = self.n_targets
            out = dict(sum_w=torch.empty(n, dtype=torch.float64, device=dev),
                       map_e=torch.empty(n, dtype=torch.float32, device=dev),
                       map_b=torch.empty(n, dtype=torch.float32, device=dev),
                       var=torch.empty(n, dtype=torch.float32, device=dev),
                       count=torch.empty(n, dtype=torch.int64, device=dev),
                       members=torch.empty(n, dtype=torch.int32, device=dev))
        n = self.n_targets
        m = N.SmartMaps(_ptr(out.get("sum_w"), torch.float64, "sum_w", n),
                        _ptr(out.get("map_e"), torch.float32, "map_e", n),
                        _ptr(out.get("map_b"), torch.float32, "map_b", n),
                        _ptr(out.get("var"), torch.float32, "var", n),
                        _ptr(out.get("count"), torch.int64, "count", n),
                        _ptr(out.get("members"), torch.int32, "members", n))
        return out, m

    def map_pixel(self, out: dict | None = None) -> dict:
        out, m = self._out(out)
        self._check(self._lib.smart_map_pixel(self._h, ctypes.byref(m)), "smart_map_pixel")
        return out

    def set_normalisation(self, mode: str):
        """'summed' (default: M = A S / sum_w) or 'averaged' (each bin pixel's shear over its own weight, times
        the pixel area)."""
        m = {"summed": 0, "averaged": 1}[mode]
        self._check(self._lib.smart_set_normalisation(self._h, m), "smart_set_normalisation")

    def map_barycentre(self, out: dict | None = None) -> dict:
        """Pixel-based map with the bin pixels at their galaxies' barycentres (needs bin_galaxies)."""
        out, m = self._out(out)
        self._check(self._lib.smart_map_barycentre(self._h, ctypes.byref(m)), "smart_map_barycentre")
        return out

    def map_bruteforce(self, out: dict | None = None) -> dict:
        out, m = self._out(out)
        self._check(self._lib.smart_map_bruteforce(self._h, ctypes.byref(m)), "smart_map_bruteforce")
        return out

    def map_projected(self, ra_c_deg: float, dec_c_deg: float, out: dict | None = None) -> dict:
        """Cartesian (projected) map about the reference point (needs bin_galaxies)."""
        out, m = self._out(out)
        self._check(self._lib.smart_map_projected(self._h, float(ra_c_deg), float(dec_c_deg), ctypes.byref(m)),
                    "smart_map_projected")
        return out

    def annulus_stats(self, ra_ref_deg: float, dec_ref_deg: float, rmax_rad: float, m_x: torch.Tensor,
                      m_ref: torch.Tensor, nbins: int) -> dict:
        """Equal-area annuli about the reference point: count, mean and sd of
        (m_x - m_ref) / sd(m_ref) per annulus (device tensors)."""
        n = self.n_targets
        dev = m_x.device
        count = torch.empty(nbins, dtype=torch.int64, device=dev)
        mean = torch.empty(nbins, dtype=torch.float64, device=dev)
        sd = torch.empty(nbins, dtype=torch.float64, device=dev)
        self._check(self._lib.smart_annulus_stats(self._h, float(ra_ref_deg), float(dec_ref_deg), float(rmax_rad),
                                                  _ptr(m_x, torch.float32, "m_x", n),
                                                  _ptr(m_ref, torch.float32, "m_ref", n), int(nbins),
                                                  _ptr(count, torch.int64, "count"), _ptr(mean, torch.float64, "mean"),
                                                  _ptr(sd, torch.float64, "sd")), "smart_annulus_stats")
        return dict(count=count, mean=mean, sd=sd)

    def sync(self, timeout_s: float = 0.0):
        self._check(self._lib.smart_sync(self._h, float(timeout_s)), "smart_sync")

    def fp64_decisions(self) -> int:
        return int(self._lib.smart_last_fp64_decisions(self._h))

    # -- kernel timing
    def timing(self, enable: bool = True):
        """Start (or stop and discard) the per-kernel event record of this context."""
        self._check(self._lib.smart_timing_enable(self._h, 1 if enable else 0), "smart_timing_enable")

    def timing_read(self, kernel: str, timeout_s: float = 60.0):
        """(launches, summed ms) of one kernel since timing(True); kernel names as in _native.KERNELS."""
        n, ms = ctypes.c_int64(), ctypes.c_double()
        self._check(self._lib.smart_timing_read(self._h, N.KERNELS[kernel], ctypes.byref(n), ctypes.byref(ms),
                                                float(timeout_s)), "smart_timing_read")
        return int(n.value), float(ms.value)

    def general_targets(self) -> torch.Tensor:
        """Positions of the targets the last pixel map sent to the general kernel (int64, device)."""
        ng = ctypes.c_int64()
        self._check(self._lib.smart_get_general_targets(self._h, None, 0, ctypes.byref(ng)),
                    "smart_get_general_targets")
        dev = torch.device("cuda", torch.cuda.current_device())
        idx = torch.empty(int(ng.value), dtype=torch.int32, device=dev)
        if idx.numel():
            self._check(self._lib.smart_get_general_targets(self._h, _ptr(idx, torch.int32, "idx"), idx.numel(),
                                                            ctypes.byref(ng)), "smart_get_general_targets")
        self.sync(60)
        return idx.long()

    def general_pairs(self):
        """The general kernel's mirror pairs: (pairs [n_pairs, 2] int64 on the
        device, target positions (lower, image)), and the number of general
        targets left unpaired."""
        npairs, nsingle = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.smart_get_general_pairs(self._h, None, 0, ctypes.byref(npairs), ctypes.byref(nsingle)),
                    "smart_get_general_pairs")
        dev = torch.device("cuda", torch.cuda.current_device())
        pairs = torch.empty((int(npairs.value), 2), dtype=torch.int32, device=dev)
        if pairs.numel():
            self._check(self._lib.smart_get_general_pairs(self._h, _ptr(pairs, torch.int32, "pairs"), pairs.shape[0],
                                                          ctypes.byref(npairs), ctypes.byref(nsingle)),
                        "smart_get_general_pairs")
        self.sync(60)
        return pairs.long(), int(nsingle.value)

    def set_band_slot_limit(self, n_slots: int):
        """Testing aid: cap the general kernel's guard-band slots (0: default)."""
        self._check(self._lib.smart_set_band_slot_limit(self._h, int(n_slots)), "smart_set_band_slot_limit")

    # -- inspection
    def get_catalog(self, n: int):
        dev = torch.device("cuda", torch.cuda.current_device())
        perm = torch.empty(n, dtype=torch.int64, device=dev)
        pix = torch.empty(n, dtype=torch.int64, device=dev)
        off = torch.empty(self.npix_bin + 1, dtype=torch.int64, device=dev)
        self._check(self._lib.smart_get_catalog(self._h, _ptr(perm, torch.int64, "perm"),
                                                _ptr(pix, torch.int64, "pix"), _ptr(off, torch.int64, "off")),
                    "smart_get_catalog")
        return perm, pix, off

    def mlp_features(self, pixel_out: dict, brute_out: dict | None = None, sum_n2: bool = False) -> dict:
        """Features [M_pix^E, sum_w, var(n_p), z] of the targets from a pixel map of this context
        (and, with a galaxy-level map of the same targets, the training target and validity)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        n = self.n_targets
        _, pm = self._out(pixel_out)
        feat = torch.empty((n, N.MLP_FEATURES), dtype=torch.float32, device=dev)
        valid = torch.empty(n, dtype=torch.uint8, device=dev)
        target = torch.empty(n, dtype=torch.float32, device=dev) if brute_out is not None else None
        n2 = torch.empty(n, dtype=torch.int64, device=dev) if sum_n2 else None
        bm = ctypes.byref(self._out(brute_out)[1]) if brute_out is not None else None
        self._check(self._lib.smart_mlp_features(self._h, ctypes.byref(pm), bm, _ptr(feat, torch.float32, "feat"),
                                                 _ptr(target, torch.float32, "target"),
                                                 _ptr(valid, torch.uint8, "valid"), _ptr(n2, torch.int64, "n2")),
                    "smart_mlp_features")
        return dict(feat=feat, target=target, valid=valid, sum_n2=n2)

    def get_binned(self):
        dev = torch.device("cuda", torch.cuda.current_device())
        m = self.npix_bin
        G1, G2, W, S2 = (torch.empty(m, dtype=torch.float32, device=dev) for _ in range(4))
        n_p = torch.empty(m, dtype=torch.int32, device=dev)
        self._check(self._lib.smart_get_binned(self._h, *(_ptr(x, x.dtype, "b") for x in (G1, G2, W, S2, n_p))),
                    "smart_get_binned")
        return dict(G1=G1, G2=G2, W=W, S2=S2, n=n_p)


class Batch:
    """Many pixel-based maps in one persistent launch replayed from a CUDA graph."""

    def __init__(self, ctxs: list, outs: list | None = None, autotune: bool = True,
                 stream: torch.cuda.Stream | None = None):
        self._lib = N.load()
        self.ctxs = list(ctxs)
        if outs is None:
            outs = [None] * len(self.ctxs)
        pairs = [c._out(o) for c, o in zip(self.ctxs, outs)]
        self.outs = [p[0] for p in pairs]
        maps = (N.SmartMaps * len(pairs))(*[p[1] for p in pairs])
        hs = (ctypes.c_void_p * len(self.ctxs))(*[c._h.value for c in self.ctxs])
        h = ctypes.c_void_p()
        st = self._lib.smart_batch_create(hs, maps, len(self.ctxs), 1 if autotune else 0,
                                          _stream_handle(stream), ctypes.byref(h))
        if st:
            msg = self._lib.smart_batch_last_error(None)
            raise SmartError(st, "smart_batch_create: " + (msg.decode() if msg else ""))
        self._h = h
        self._maps = maps

    def run(self):
        st = self._lib.smart_batch_run(self._h)
        if st:
            raise SmartError(st, "smart_batch_run: " + (self._lib.smart_batch_last_error(self._h) or b"").decode())
        return self.outs

    def info(self) -> dict:
        cps, lf, ni, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_double()
        self._lib.smart_batch_info(self._h, ctypes.byref(cps), ctypes.byref(lf), ctypes.byref(ni), ctypes.byref(ms))
        return dict(ctas_per_sm=cps.value, longest_first=bool(lf.value), n_items=ni.value, tuned_ms=ms.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.smart_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Residual:
    """Learned residual correction of the pixel-based map (bf16 tensor-core
    network, or the float32 checking mode)."""

    def __init__(self, precision: str = "bf16", stream: torch.cuda.Stream | None = None):
        self._lib = N.load()
        prec = {"bf16": N.MLP_BF16, "fp32": N.MLP_FP32}[precision]
        h = ctypes.c_void_p()
        st = self._lib.smart_mlp_create(prec, _stream_handle(stream), ctypes.byref(h))
        if st:
            raise SmartError(st, "smart_mlp_create")
        self._h = h
        self.precision = precision

    def _check(self, st: int, what: str):
        if st:
            msg = self._lib.smart_mlp_last_error(self._h)
            raise SmartError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.smart_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters and standardisation (host arrays)
    def set_params(self, params: torch.Tensor):
        p = params.detach().to("cpu", torch.float32).contiguous()
        if p.numel() != N.MLP_NPARAMS:
            raise ValueError(f"expected {N.MLP_NPARAMS} parameters")
        self._check(self._lib.smart_mlp_set_params(self._h, ctypes.c_void_p(p.data_ptr())), "smart_mlp_set_params")

    def get_params(self) -> torch.Tensor:
        p = torch.empty(N.MLP_NPARAMS, dtype=torch.float32)
        self._check(self._lib.smart_mlp_get_params(self._h, ctypes.c_void_p(p.data_ptr())), "smart_mlp_get_params")
        return p

    def set_scaler(self, scaler):
        a = (ctypes.c_double * 10)(*[float(x) for x in scaler])
        self._check(self._lib.smart_mlp_set_scaler(self._h, a), "smart_mlp_set_scaler")

    def get_scaler(self) -> list:
        a = (ctypes.c_double * 10)()
        self._check(self._lib.smart_mlp_get_scaler(self._h, a), "smart_mlp_get_scaler")
        return list(a)

    def fit_scaler(self, feat: torch.Tensor, target: torch.Tensor, rows: torch.Tensor | None = None):
        n = rows.numel() if rows is not None else target.numel()
        self._check(self._lib.smart_mlp_fit_scaler(self._h, _ptr(feat, torch.float32, "feat"),
                                                   _ptr(target, torch.float32, "target"),
                                                   _ptr(rows, torch.int32, "rows"), n), "smart_mlp_fit_scaler")

    # -- training
    def gradient(self, feat, target, idx=None, batch: int | None = None) -> torch.Tensor:
        """Gradient of the batch's mean squared error; the last entry is the sum of squared errors."""
        n = idx.numel() if idx is not None else (batch if batch is not None else target.numel())
        g = torch.empty(N.MLP_NPARAMS + 1, dtype=torch.float32, device=feat.device)
        self._check(self._lib.smart_mlp_gradient(self._h, _ptr(feat, torch.float32, "feat"),
                                                 _ptr(target, torch.float32, "target"), _ptr(idx, torch.int32, "idx"),
                                                 n, _ptr(g, torch.float32, "grad")), "smart_mlp_gradient")
        return g

    def train_step(self, feat, target, idx, lr: float, loss_out: torch.Tensor | None = None):
        self._check(self._lib.smart_mlp_train_step(self._h, _ptr(feat, torch.float32, "feat"),
                                                   _ptr(target, torch.float32, "target"),
                                                   _ptr(idx, torch.int32, "idx"), idx.numel(), float(lr),
                                                   _ptr(loss_out, torch.float32, "loss")), "smart_mlp_train_step")

    @property
    def step(self) -> int:
        return int(self._lib.smart_mlp_step(self._h))

    def sync(self, timeout_s: float = 0.0):
        self._check(self._lib.smart_mlp_sync(self._h, float(timeout_s)), "smart_mlp_sync")

    # -- inference
    def infer(self, feat: torch.Tensor, plain: torch.Tensor, out: torch.Tensor | None = None,
              correction: torch.Tensor | None = None, n_fallback: torch.Tensor | None = None) -> torch.Tensor:
        n = plain.numel()
        if out is None:
            out = torch.empty_like(plain)
        self._check(self._lib.smart_mlp_infer(self._h, _ptr(feat, torch.float32, "feat", 4 * n),
                                              _ptr(plain, torch.float32, "plain"), n,
                                              _ptr(out, torch.float32, "out", n),
                                              _ptr(correction, torch.float32, "correction", n),
                                              _ptr(n_fallback, torch.int64, "n_fallback", 1)), "smart_mlp_infer")
        return out

    # -- checkpoint
    def state(self) -> bytes:
        size = ctypes.c_int64()
        self._check(self._lib.smart_mlp_get_state(self._h, None, 0, ctypes.byref(size)), "smart_mlp_get_state")
        buf = ctypes.create_string_buffer(size.value)
        self._check(self._lib.smart_mlp_get_state(self._h, buf, size.value, ctypes.byref(size)), "smart_mlp_get_state")
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._check(self._lib.smart_mlp_set_state(self._h, buf, len(blob)), "smart_mlp_set_state")

    def save(self, path: str):
        with open(path, "wb") as f:
            f.write(self.state())

    def load(self, path: str):
        with open(path, "rb") as f:
            self.load_state(f.read())
