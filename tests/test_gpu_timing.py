"""Per-kernel timing record and the general-target query of the library."""
import numpy as np
import pytest
import torch

from paper_2609_11181_b300 import api

from _cases import binned_field_oracle, catalog, cap_targets

pytestmark = pytest.mark.gpu


def test_pixel_timing_and_general_targets(cuda_device):
    # a cap reaching the polar rings: both pixel kernels run
    nside = 256
    b, foot = binned_field_oracle(21, nside, 30.0, 40.0, 12.0, mean_count=10.0)
    tg = torch.from_numpy(np.nonzero(foot)[0].astype(np.int64)).to(cuda_device)
    ctx = api.Context(nside, 30.0, "schirmer", nside_bin=nside)
    ctx.set_targets(tg)
    ctx.set_binned(*(x.to(cuda_device) for x in (b.G1, b.G2, b.W, b.S2, b.n)))
    ctx.timing(True)
    for _ in range(3):
        ctx.map_pixel()
    ctx.sync(60)
    nt, mt = ctx.timing_read("pixel_toeplitz")
    ng, mg = ctx.timing_read("pixel_general")
    gen = ctx.general_targets()
    assert 0 < gen.numel() < tg.numel()
    assert nt == 3 and ng == 3 and mt > 0 and mg > 0
    g = gen.cpu().numpy()
    assert np.unique(g).size == g.size and g.min() >= 0 and g.max() < tg.numel()
    # the general kernel takes whole output rings: every target of a listed ring is listed
    ring_of = lambda p: np.searchsorted(np.cumsum([0] + [4 * min(i, nside, 4 * nside - i) for i in range(1, 4 * nside)]),
                                        p, side="right")
    rings = ring_of(tg.cpu().numpy())
    listed = np.zeros(tg.numel(), bool)
    listed[g] = True
    for r in np.unique(rings[listed]):
        assert listed[rings == r].all()
    ctx.timing(False)
    ctx.map_pixel()
    ctx.sync(60)
    assert ctx.timing_read("pixel_toeplitz")[0] == 0


def test_bruteforce_and_binning_timing(cuda_device):
    cat = catalog(22, 50_000, 120.0, -10.0, 3.0)
    ctx = api.Context(128, 20.0, "poly", nside_bin=512)
    ctx.set_targets(torch.from_numpy(cap_targets(128, 120.0, -10.0, 2.0)).to(cuda_device))
    ctx.timing(True)
    c = cat.to(cuda_device)
    ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
    ctx.map_bruteforce()
    ctx.sync(60)
    for name in ("bin_keys", "bin_sort", "bin_records", "bin_pixel_sums", "galaxy", "galaxy_band",
                 "galaxy_finalise"):
        n, ms = ctx.timing_read(name)
        assert n == 1 and ms >= 0.0, name


def test_sync_deadline_times_out_and_context_stays_usable(cuda_device):
    # a stream kept busy by several maps: a wait with a tiny deadline gives up
    # with SMART_E_TIMEOUT; the work completes and a later wait succeeds
    from paper_2609_11181_b300 import workloads
    wl = workloads.pixel_workload(cuda_device, api.pix2vec, nside=1024, area_deg2=2000.0, theta_ap=30.0,
                                  filt="schirmer", dec0=50.0)
    ctx = api.Context(wl.nside, wl.theta_ap_arcmin, wl.filter, nside_bin=wl.nside)
    ctx.set_targets(wl.targets)
    ctx.set_binned(wl.G1, wl.G2, wl.W, wl.S2, wl.n)
    ref = ctx.map_pixel()
    ctx.sync(60)
    ref = {k: v.clone() for k, v in ref.items()}
    out = None
    for _ in range(8):
        out = ctx.map_pixel()
    with pytest.raises(api.SmartError) as err:
        ctx.sync(1e-6)
    assert "TIMEOUT" in str(err.value)
    ctx.sync(60)
    for k in ref:
        assert torch.equal(out[k], ref[k]), k


def test_map_calls_return_before_the_work_completes(cuda_device):
    """The boundary's map calls only enqueue work: with the context stream
    held by a long probe kernel, smart_bin_galaxies and every map call return
    at once (the stream is still busy afterwards), smart_sync then waits, and
    the maps equal those of a quiet stream."""
    import time
    cat = catalog(23, 80_000, 200.0, 35.0, 4.0, w_range=(0.5, 1.5))
    tg = torch.from_numpy(cap_targets(256, 200.0, 35.0, 3.0)).to(cuda_device)
    c = cat.to(cuda_device)

    def run(busy):
        ctx = api.Context(256, 20.0, "schirmer", nside_bin=512)
        ctx.set_targets(tg)                 # set-up: builds the tables (may wait)
        if busy:
            api.fma_probe(32, 1 << 20, 8)   # 8e13 flop: about 1.1 s of FMA work on the same stream
        t0 = time.perf_counter()
        ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
        outs = [ctx.map_bruteforce(), ctx.map_pixel(), ctx.map_barycentre(), ctx.map_projected(200.0, 35.0)]
        dt = time.perf_counter() - t0
        pending = not torch.cuda.current_stream().query()
        ctx.sync(120)
        res = [{k: v.clone() for k, v in o.items()} for o in outs]
        ctx.close()
        return dt, pending, res

    # the quiet run first: the first launch of a kernel in a process may wait
    # while the driver loads it (and sizes its local memory)
    _, _, quiet_maps = run(False)
    dt, pending, busy_maps = run(True)
    assert pending, "the stream was idle right after the calls: some call waited"
    assert dt < 0.25, f"the calls took {dt:.3f} s on a busy stream"
    for a, b in zip(busy_maps, quiet_maps):
        for k in a:
            assert torch.equal(a[k], b[k]), k


def test_fma_probe_forms(cuda_device):
    """The probe's three forms run and count their operations: 2 x CTAs x 256
    threads x iters x 128 FMAs, twice that for the packed float32 pairs."""
    nsm = torch.cuda.get_device_properties(cuda_device).multi_processor_count
    base = 2.0 * nsm * 2 * 256 * 64 * 128
    assert api.fma_probe(32, 64, 2) == base
    assert api.fma_probe(64, 64, 2) == base
    assert api.fma_probe(32, 64, 2, packed=True) == 2 * base
    torch.cuda.synchronize()
