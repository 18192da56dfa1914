"""Benchmark of the SMART aperture-mass hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--workload pixel4096|brute2048]

Default workload (N=1): the NSIDE-4096 pixel-based map over a 15,000 deg^2
cap (binned shear given per pixel, Schirmer filter x_c = 0.15, theta_ap =
10').  After the headline, the default single-GPU run also times the other
forms of the metric at their own configurations (brute force over 5e7
galaxies, 64 maps in one batched launch, the learned correction and the
barycentre form) and reports them under "forms"; --no-forms skips them.  A step is one full pixel-based map: register the binned input and run
the aperture kernel (geometry, membership, rotation, filter, compensated sums
and the summed normalisation all happen in that launch).  The metric is
pairs per second (Gpair/s) -- a pair is one (target pixel, pixel whose
centre lies within theta_ap) -- with the map time in ms_per_step.

Inputs (4 GB of full-sky binned arrays) are larger than L2, so no flush is
needed between steps.  For N > 1 (torchrun), each rank computes an
independent replica (the path is not sharded): value = pairs of all ranks /
max time.

``--impl reference`` times the float64 CPU oracle on a bounded random sample
of the same targets on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_11181_b300 import api, workloads  # noqa: E402

METRIC = "NSIDE-4096 M_ap map time & Gpair/s, chosen vs plain form at <=1e-4 rel err"
FP32_NOMINAL_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12     # 148 SMs x 128 FP32 lanes x FMA x 2032 MHz
# Algorithmic float32 work of one member pair in the direct form of the method
# (FMA = 2 flop): the ring-pair geometry with no sqrt, divide or trig (azimuth
# offset, sine and haversine of it, chord^2 = A + B h, tangent-plane direction
# x, y), cos 2psi and sin 2psi from x and y, the filter weight, the rotation
# into gamma_+ and gamma_x, and the E, B, variance and weight sums: about 45
# flop for the polynomial filter; a tabulated filter (Schirmer, Jarvis) adds
# one reciprocal square root and a cubic table lookup (about 9 more).
ALGO_FLOPS_PER_PAIR = {"poly": 45, "schirmer": 54, "jarvis": 54}
# Executed float32 work per pair of the Toeplitz kernel: geometry, filter and
# rotation are tabulated once per ring pair and index offset and shared by
# every target, so a pair costs 4 FMAs for E and B, 1 FMA for the variance and
# one add for the weight.
TOEPLITZ_EXEC_FLOPS_PER_PAIR = 11
# Executed float32 work per pair of the general pixel kernel: 49 measured with
# a tabulated filter (ncu: fadd + fmul + 2 ffma thread instructions per pair,
# NSIDE 2048 case), matching the pair body's count (FMA = 2, a hardware square
# root or reciprocal = 1): lattice offset 3, sine / haversine series 7, chord
# 2, tangent-plane direction and cos / sin 2psi 10, E / B 10, variance and
# weight sums 4, table 9, weight 5; the polynomial filter replaces table and
# weight (14) by the chord-to-separation series, Q and Q / sin^2 d (18).
GENERAL_EXEC_FLOPS_PER_PAIR = {"schirmer": 49, "jarvis": 49, "poly": 53}
# The same for a general target that runs with its mirror image (one thread
# for both; the image's pairs have the target's geometry with x -> -x): the
# geometry, filter and weight of a pair (36 flop with a table, 40 with the
# polynomial filter, as counted above) serve two pairs, each of which adds
# its E / B, variance and weight sums and shares Q^2 and the weighted
# rotation terms Q cos 2psi, Q sin 2psi: 30 measured with a tabulated filter
# (ncu, as above, NSIDE 2048 case), 32 polynomial (the count's difference of
# 4 per two pairs added).
GENERAL_PAIRED_EXEC_FLOPS_PER_PAIR = {"schirmer": 30, "jarvis": 30, "poly": 32}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu_index: int):
        self.proc = None
        out_dir = os.environ.get("SMART_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"smart_clocks_rank{gpu_index}_{os.getpid()}.csv")
        exe = shutil.which("nvidia-smi")
        if exe is None:
            return
        os.makedirs(out_dir, exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.f = open(self.path, "w")
        self.proc = subprocess.Popen([exe, f"--id={gpu_index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                      "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x: float, op_name: str) -> float:
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"     # gloo reduces host tensors
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(x: float, world: int) -> float:
    return x if world == 1 else _reduce(x, "MAX")


def sum_over_ranks(x: float, world: int) -> float:
    return x if world == 1 else _reduce(x, "SUM")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            return None
    return None


SCAN_TILE = 2048          # elements per block of the library's exclusive scan


def scan_launches(n: int) -> int:
    """Kernel launches of the library's exclusive scan over n elements: one
    tile pass, a scan of the block sums (recursively), one add pass."""
    if n <= 0:
        return 0
    nb = -(-n // SCAN_TILE)
    return 1 if nb == 1 else 2 + scan_launches(nb)


def _sha256(paths):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` at `workload` from the committed ncu
    summary profiles/<kernel>_<workload>.md, or None when there is none or
    when the kernel's sources changed since the counters were taken (the
    summary records the sha256 of the source files it covers)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.lstrip().startswith("- "):
            k, v = line.lstrip()[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    try:
        srcs = fields["sources"].split()
        if _sha256(srcs) != fields["source_sha256"]:
            return None
        return int(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError, OSError):
        return None


def measure_fma_peaks(stream, target_ms=60.0, repeats=3):
    """FP32 and FP64 FMA throughput of this GPU (TFLOP/s), measured with the
    library's probe kernel (eight FMA chains per thread, 8 CTAs of 256
    threads per SM) timed with CUDA events on `stream`; best of `repeats`
    launches of about target_ms each after a warm-up.  Changes no clock or
    power setting."""
    out = {}
    for bits, packed, key in ((32, False, "fp32"), (32, True, "fp32x2"), (64, False, "fp64")):
        iters = 512 if bits == 32 else 16
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        while True:                                   # size the launch to about target_ms
            a.record(stream)
            flops = api.fma_probe(bits, iters, 8, stream, packed)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            if ms >= 0.25 * target_ms or iters > (1 << 26):
                break
            iters *= 4
        iters = max(1, int(iters * target_ms / max(ms, 1e-3)))
        best = 0.0
        for _ in range(repeats):
            a.record(stream)
            flops = api.fma_probe(bits, iters, 8, stream, packed)
            b.record(stream)
            b.synchronize()
            best = max(best, flops / (a.elapsed_time(b) * 1e-3) / 1e12)
        out[f"{key}_tflops"] = round(best, 3)
    out["how"] = ("library probe smart_fma_probe: 8 independent FMA chains per thread, 8 x 256-thread CTAs per SM, "
                  f"about {target_ms:.0f} ms per launch, best of {repeats} (CUDA events)")
    out["fp32_nominal_tflops"] = round(FP32_NOMINAL_TFLOPS, 2)
    return out


def fp32_peak(peaks_live):
    """The FP32 roofline denominator: the higher of the scalar and the packed
    (two FMAs per instruction) probe rates, and where it comes from."""
    sc, pk = peaks_live["fp32_tflops"], peaks_live.get("fp32x2_tflops", 0.0)
    src = (f"FP32 FMA throughput measured in this run by the library's probe ({peaks_live['how']}): "
           f"scalar FMA {sc}, packed two-lane FMA {pk}; the higher is the peak; "
           f"nominal {FP32_NOMINAL_TFLOPS:.2f} (148 SMs x 128 lanes x 2 x 2032 MHz)")
    return max(sc, pk), src


def kernel_roofline(ctx, kernels: dict, workload: str, peak_tflops: float, peak_source: str):
    """Roofline of the dominant kernel from the context's per-launch events.

    kernels: {name: (pairs per launch, algorithmic flops per pair, executed
    flops per pair, kernel symbol, shares work between pairs)}.  The dominant
    kernel is the one with the largest summed time over the timed steps;
    achieved = algorithmic flops per launch (the direct-form count per pair x
    member pairs) / its mean launch time, except for a kernel that shares work
    between pairs (the Toeplitz kernel: one geometry entry serves every target
    at the same ring offset; the general kernel with mirror pairs: one
    geometry evaluation serves a target and its image), which is held to the
    flops it executes.  Both figures are reported per kernel."""
    per = {}
    for name, (pairs, fpp, exec_fpp, sym, shares) in kernels.items():
        n, ms = ctx.timing_read(name)
        if n == 0:
            continue
        t = ms / n * 1e-3
        per[name] = {"kernel": sym, "launches": n, "total_ms": round(ms, 3), "ms_per_launch": round(ms / n, 4),
                     "pairs_per_launch": int(pairs), "gpair_s": round(pairs / t / 1e9, 2) if t > 0 else None,
                     "algorithmic_flops_per_pair": fpp, "executed_flops_per_pair": exec_fpp,
                     "shares_work_between_pairs": shares,
                     "algorithmic_tflops": round(pairs * fpp / t / 1e12, 2) if t > 0 and fpp else None,
                     "executed_tflops": round(pairs * exec_fpp / t / 1e12, 2) if t > 0 and exec_fpp else None}
    if not per:
        return None, per
    dom = max(per, key=lambda k: per[k]["total_ms"])
    d = per[dom]
    if not d["shares_work_between_pairs"]:
        achieved, basis = d["algorithmic_tflops"], "algorithmic flops (direct form per member pair)"
    else:
        achieved, basis = d["executed_tflops"], "executed flops (work shared between pairs)"
    roof = {"bound": "alu", "achieved": achieved, "peak": round(peak_tflops, 2), "unit": "TFLOP/s",
            "frac": round(achieved / peak_tflops, 4), "traffic": profiled_traffic(d["kernel"], workload),
            "kernel": d["kernel"], "launches": d["launches"], "ms_per_launch": d["ms_per_launch"],
            "pairs_per_launch": d["pairs_per_launch"],
            "algorithmic_flops_per_pair": d["algorithmic_flops_per_pair"],
            "executed_flops_per_pair": d["executed_flops_per_pair"], "achieved_basis": basis,
            "peak_source": peak_source}
    return roof, per


# ---------------------------------------------------------------------------
# CPU baseline: the float64 oracle on a bounded sample of the same targets
# ---------------------------------------------------------------------------
def cpu_baseline_pixel(wl, G, budget_s=15.0, seed=0, return_sample=False):
    """G: host copies of (G1, G2, W, S2, n).  With return_sample, also the
    sampled targets and the oracle's sums for them."""
    import oracle
    tg = wl.targets.cpu().numpy()
    rng = np.random.default_rng(seed)
    kind = 2 if wl.filter == "schirmer" else 1
    th = wl.theta_ap_arcmin * math.pi / 10800
    cores = os.cpu_count() or 1

    def run(m):
        s = np.sort(rng.choice(tg, size=min(m, tg.size), replace=False))
        cv = oracle.pix2vec(wl.nside, s)
        t0 = time.perf_counter()
        r = oracle.aperture_pixels_f32(cv, wl.nside, *G, kind, th)
        return time.perf_counter() - t0, int(r["NPIX"].sum()), s.size, (s, r)

    m = max(256, cores * 64)
    dt, pairs, m, sr = run(m)
    while dt < 0.25 * budget_s and m < tg.size:          # grow until the timing is meaningful
        m = int(min(tg.size, m * max(2.0, 0.5 * budget_s / max(dt, 1e-3))))
        dt, pairs, m, sr = run(m)
    cb = {"value": pairs / dt / 1e9, "unit": "Gpair/s", "cores": cores, "kind": "oracle",
          "sample": f"{m} random targets of {tg.size} (float64 oracle, OpenMP over targets), {pairs} pairs, "
                    f"{dt:.1f} s"}
    if return_sample:
        return cb, pairs, dt, m, sr
    return cb, pairs, dt, m


def accuracy_vs_oracle(out: dict, targets: np.ndarray, sample: np.ndarray, ref: dict, theta_ap: float,
                       tol: float = 1e-4) -> dict:
    """The map at the sampled targets against the float64 oracle's sums for
    them: counts bit-exact, rms(M - M_oracle) / rms(M_oracle) for M_E, M_B
    and sigma^2, largest relative error of the weight sum."""
    import oracle
    idx = np.searchsorted(targets, sample)
    assert np.array_equal(targets[idx], sample)
    ref = oracle.finalise(ref, theta_ap)
    it = torch.from_numpy(idx).to(out["map_e"].device)
    got = {k: v[it].cpu().numpy() for k, v in out.items()}
    rr = {k: oracle.rms_rel(got[g].astype(np.float64), ref[o])
          for k, g, o in (("map_e", "map_e", "ME"), ("map_b", "map_b", "MB"), ("var", "var", "VAR"))}
    sw = float(np.max(np.abs(got["sum_w"] - ref["SW"]) / np.maximum(np.abs(ref["SW"]), 1e-300)))
    counts = bool(np.array_equal(got["count"], ref["N"]))
    if "members" in got and "NPIX" in ref:
        counts = counts and bool(np.array_equal(got["members"], ref["NPIX"]))
    return {"targets": int(sample.size), "counts_bit_exact": counts,
            "rms_rel": {k: float(f"{v:.3e}") for k, v in rr.items()}, "sum_w_max_rel": float(f"{sw:.3e}"),
            "tolerance": tol, "within_tolerance": counts and all(v <= tol for v in rr.values()) and sw <= 1e-6}


PIXEL_WORKLOADS = workloads.PIXEL_WORKLOADS


def _oracle_centres(nside, p):
    """Pixel centres from the float64 oracle, for inputs that the oracle leg
    also consumes (no oracle input may come from the CUDA path)."""
    import oracle
    return torch.from_numpy(oracle.pix2vec(nside, p.cpu().numpy())).to(p.device)


def first_map_ms(wl, inputs, out):
    """A one-shot caller's map: a fresh context, targets, the binned input and
    one pixel map, synchronised (host clock around everything, so the
    context's table set-up and its allocations are included)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c = api.Context(wl.nside, wl.theta_ap_arcmin, wl.filter, nside_bin=wl.nside)
    c.set_targets(wl.targets)
    c.set_binned_packed(*inputs)
    c.map_pixel(out)
    c.sync(300)
    ms = (time.perf_counter() - t0) * 1e3
    c.close()
    return ms


def run_native_pixel(args, world, rank):
    dev = torch.device("cuda", torch.cuda.current_device())
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    stream = torch.cuda.current_stream()
    peaks_live = measure_fma_peaks(stream)
    t_gen = time.perf_counter()
    # the oracle leg compares the map with float64 sums over the same inputs,
    # so those inputs are generated with the oracle's pixel centres
    wl = workloads.pixel_workload(dev, _oracle_centres if want_cpu else api.pix2vec,
                                  **PIXEL_WORKLOADS[args.workload])
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    ctx = api.Context(wl.nside, wl.theta_ap_arcmin, wl.filter, nside_bin=wl.nside)
    ctx.set_targets(wl.targets)
    n = wl.targets.numel()
    out = ctx._out(None)[0]
    host_G = [x.cpu().numpy() for x in (wl.G1, wl.G2, wl.W, wl.S2, wl.n)] if want_cpu else None
    # the library's native input layout: (G1, G2, S2, W) per pixel + counts
    px = torch.stack([wl.G1, wl.G2, wl.S2, wl.W], dim=1).contiguous()
    inputs = (px, wl.n)
    del wl.G1, wl.G2, wl.S2, wl.W

    def step():
        ctx.set_binned_packed(*inputs)
        ctx.map_pixel(out)

    # a one-shot map first, on a fresh context (tables built, nothing cached)
    scratch_out = ctx._out(None)[0]
    first_ms = first_map_ms(wl, inputs, scratch_out)
    del scratch_out
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    members = out["members"].long()
    pairs_step = int(members.sum().item())
    gen_idx = ctx.general_targets()
    pairs_gen = int(members[gen_idx].sum().item()) if gen_idx.numel() else 0
    gen_pairs, gen_single = ctx.general_pairs()
    pairs_mirror = int(members[gen_pairs.reshape(-1)].sum().item()) if gen_pairs.numel() else 0
    # launches per map: the mirror pairs (with up to a sixteenth as many
    # unpaired targets run ahead of them), else the unpaired targets alone
    npg = int(gen_pairs.shape[0])
    gen_launches = int(npg > 0) + int(gen_single > 0 and not (npg > 0 and 16 * gen_single <= npg))
    gen_exec = ((pairs_mirror * GENERAL_PAIRED_EXEC_FLOPS_PER_PAIR[wl.filter]
                 + (pairs_gen - pairs_mirror) * GENERAL_EXEC_FLOPS_PER_PAIR[wl.filter]) / pairs_gen
                if pairs_gen else GENERAL_EXEC_FLOPS_PER_PAIR[wl.filter])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(torch.cuda.current_device())
    barrier(world)
    torch.cuda.synchronize()
    ctx.timing(True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ck = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = max_over_ranks(total_ms / args.steps, world)
    pairs_all = sum_over_ranks(float(pairs_step), world)
    value = pairs_all / (ms_step * 1e-3) / 1e9
    algo = ALGO_FLOPS_PER_PAIR[wl.filter]
    peak, peak_src = fp32_peak(peaks_live)
    roof, per_kernel = kernel_roofline(
        ctx, {"pixel_toeplitz": (pairs_step - pairs_gen, algo, TOEPLITZ_EXEC_FLOPS_PER_PAIR, "k_pixel_toeplitz", True),
              "pixel_general": (pairs_gen, algo, round(gen_exec, 1), "k_pixel_general", pairs_mirror > 0),
              "pixel_band": (0, None, None, "k_pixel_band", False)},
        args.workload, peak, peak_src)
    ctx.timing(False)
    npix_bin = 12 * wl.nside ** 2
    # the general timer spans the mirror-pair and the unpaired launch of a map
    launches_step = (sum(v["launches"] for v in per_kernel.values()) / args.steps + scan_launches(npix_bin + 1)
                     + (gen_launches - 1 if "pixel_general" in per_kernel else 0))
    map_roof = {"achieved": round(pairs_step * algo / (ms_step * 1e-3) / 1e12, 2), "unit": "TFLOP/s",
                "peak": peak, "frac": round(pairs_step * algo / (ms_step * 1e-3) / 1e12 / peak, 4),
                "basis": f"whole step: member pairs x {algo} algorithmic flop per pair / ms_per_step"}

    # end to end through the public API: every step copies its inputs from
    # pinned host memory, maps them and reads the maps back.  The input is the
    # footprint's pixels only, as runs of consecutive RING pixels
    # (smart_set_binned_runs; outside the footprint the binned data are zero,
    # so the maps equal the device run's bit for bit); the results read back
    # are the maps of the method, M_E, M_B and sigma^2 (the weight sums stay
    # on the device: copies in the two directions share the host link's
    # bandwidth).  Steps are pipelined the way a serving loop would run them:
    # double-buffered device inputs and outputs, host->device copies on one
    # stream, the map on the context's stream, device->host copies on a
    # third.  An input buffer is free again as soon as smart_set_binned_runs
    # has copied it into the context's map, so step k + 1's copy in and step
    # k - 1's copy out overlap step k's map.
    foot = wl.targets.cpu().numpy()                  # the footprint's pixels (where the data are)
    brk = np.nonzero(np.diff(foot) != 1)[0] + 1
    r_first = np.concatenate([[0], brk])
    r_end = np.concatenate([brk, [foot.size]])
    runs_np = np.stack([foot[r_first], r_end - r_first, r_first], 1).astype(np.int64)
    fidx = wl.targets
    host_in = [inputs[0][fidx].cpu().pin_memory(), inputs[1][fidx].cpu().pin_memory(),
               torch.from_numpy(runs_np).pin_memory()]
    h2d = sum(x.numel() * x.element_size() for x in host_in)
    read_back = ("map_e", "map_b", "var")
    d2h = sum(out[k].numel() * out[k].element_size() for k in read_back)
    s_in, s_map, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ectx = api.Context(wl.nside, wl.theta_ap_arcmin, wl.filter, nside_bin=wl.nside, stream=s_map)
    ectx.set_targets(wl.targets)
    dev_in = [[torch.empty(x.shape, dtype=x.dtype, device=dev) for x in host_in] for _ in range(2)]
    outs = [ectx._out(None)[0] for _ in range(2)]
    host_out = [{k: torch.empty(out[k].shape, dtype=out[k].dtype, pin_memory=True) for k in read_back}
                for _ in range(2)]
    e_steps = max(8, min(2 * args.steps, 16))          # a pipeline: fill and drain are paid once
    ev_in = [torch.cuda.Event() for _ in range(e_steps)]
    ev_set = [torch.cuda.Event() for _ in range(e_steps)]
    ev_map = [torch.cuda.Event() for _ in range(e_steps)]
    ev_out = [torch.cuda.Event() for _ in range(e_steps)]

    def e2e_run(n):
        for k in range(n):
            i = k % 2
            if k >= 2:
                # inputs of buffer i no longer read: smart_set_binned_runs has
                # copied them into the context's map
                s_in.wait_event(ev_set[k - 2])
            with torch.cuda.stream(s_in):
                for d, h in zip(dev_in[i], host_in):
                    d.copy_(h, non_blocking=True)
                ev_in[k].record(s_in)
            s_map.wait_event(ev_in[k])
            if k >= 2:
                s_map.wait_event(ev_out[k - 2])       # outputs of buffer i read back
            ectx.set_binned_runs(*dev_in[i])
            ev_set[k].record(s_map)
            ectx.map_pixel(outs[i])
            ev_map[k].record(s_map)
            s_out.wait_event(ev_map[k])
            with torch.cuda.stream(s_out):
                for key in read_back:
                    host_out[i][key].copy_(outs[i][key], non_blocking=True)
                ev_out[k].record(s_out)
        stream.wait_event(ev_out[n - 1])
        stream.wait_event(ev_map[n - 1])

    e2e_run(2)                                        # warm (tables of the second context)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    t0.record(stream)
    e2e_run(e_steps)
    t1.record(stream)
    torch.cuda.synchronize()
    same = all(torch.equal(host_out[(e_steps - 1) % 2][k].to(out[k].device), out[k]) for k in read_back)
    ectx.close()
    del dev_in, outs, host_out, host_in
    e2e_ms = max_over_ranks(t0.elapsed_time(t1) / e_steps, world)

    peaks = load_peaks()
    kmean = statistics.mean(kern_ms)
    res = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gpair/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl.desc, "targets": n, "pairs_per_step": pairs_step,
                   "nside": wl.nside, "theta_ap_arcmin": wl.theta_ap_arcmin, "filter": wl.filter,
                   "l2": f"inputs ({sum(x.numel() * x.element_size() for x in inputs) / 1e9:.1f} GB full-sky binned "
                         "arrays) larger than L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "map_time_ms": round(ms_step, 3),
        "step_ms_mean": round(kmean, 3),
        "first_map_ms": round(first_ms, 3),
        "roofline": roof,
        "map_roofline": map_roof,
        "kernels": per_kernel,
        "general_mirror_pairs": {"pairs": int(gen_pairs.shape[0]), "unpaired_targets": gen_single,
                                 "member_pairs_of_paired_targets": pairs_mirror,
                                 "member_pairs_general": pairs_gen, "launches_per_map": gen_launches},
        "fma_peaks_measured": peaks_live,
        "e2e": {"value": round(pairs_all / (e2e_ms * 1e-3) / 1e9, 3), "unit": "Gpair/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3),
                "steps": e_steps, "pipelined": "double-buffered; copy in, map and copy out on three streams",
                "input": f"footprint pixels as {len(runs_np)} runs of RING pixels (smart_set_binned_runs), "
                         f"{foot.size} of {12 * wl.nside ** 2} pixels",
                "read_back": list(read_back), "results_equal_device_run": same},
        "gpu_launches": int(round(launches_step * args.steps)),
        "clocks": ck,
        "input_gen_s": round(t_gen, 1),
    }
    if peaks:
        res["measured_peaks_present"] = True
    if want_cpu:
        cb, _, _, _, (smp, ref) = cpu_baseline_pixel(wl, host_G, return_sample=True)
        res["cpu_baseline"] = cb
        res["accuracy"] = accuracy_vs_oracle(out, wl.targets.cpu().numpy(), smp, ref,
                                             wl.theta_ap_arcmin * math.pi / 10800)
        res["accuracy"]["of"] = "the timed map (last step) at the cpu_baseline sample of targets, float64 oracle"
    ctx.close()
    del out, inputs, px
    torch.cuda.empty_cache()
    return res


GALAXY_WORKLOADS = workloads.GALAXY_WORKLOADS
# executed float32 flops per member pair of the brute-force kernel: 75
# measured for the polynomial filter (ncu: fadd + fmul + 2 ffma thread
# instructions per member pair, 4e6-galaxy case): every galaxy of the union of
# the four targets' windows is evaluated for all four (about 1.4 pairs per
# member pair), plus each galaxy's set-up; a tabulated filter adds about 6 per
# evaluated pair (table lookup and a division instead of the polynomial's
# division-free weight)
BRUTE_EXEC_FLOPS_PER_PAIR = {"poly": 75, "schirmer": 83, "jarvis": 83}


def projected_leg(ctx, wl, cat, out_sph, steps, accuracy_targets):
    """The Cartesian (projected) form, projS_pos, on the same catalogue and
    targets: gnomonic projection about the cap centre, brute force in the
    plane; its time, its accuracy against the float64 oracle, and the
    equal-area annulus statistics of (projected - spherical) / sd(spherical)
    against the distance from the projection centre (Sect. 5.2.2)."""
    stream = torch.cuda.current_stream()
    ra_c, dec_c = 0.0, 0.0
    proj = ctx.map_projected(ra_c, dec_c)            # warm
    torch.cuda.synchronize()
    ctx.timing(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        ctx.map_projected(ra_c, dec_c, proj)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    phases = {}
    for name in ("proj_records", "proj_map", "proj_band"):
        nl, t = ctx.timing_read(name)
        if nl:
            phases[name] = round(t / nl, 4)
    ctx.timing(False)
    pairs = int(proj["members"].long().sum().item())
    radius = synth_cap_radius(1000.0)
    nb = 10
    st = ctx.annulus_stats(ra_c, dec_c, radius, proj["map_e"], out_sph["map_e"], nb)
    torch.cuda.synchronize()
    edges = [math.degrees(math.acos(1 - (k / nb) * (1 - math.cos(radius)))) for k in range(nb + 1)]
    res = {"ms_per_map": round(ms, 3), "gpair_s": round(pairs / (ms * 1e-3) / 1e9, 3), "pairs": pairs,
           "phases_ms": phases, "reference_point_deg": [ra_c, dec_c],
           "annuli_vs_spherical": {"outer_radius_deg": [round(e, 3) for e in edges[1:]],
                                   "count": st["count"].cpu().tolist(),
                                   "eps_sd": [float(f"{v:.4e}") for v in st["sd"].cpu().tolist()],
                                   "eps_mean": [float(f"{v:.4e}") for v in st["mean"].cpu().tolist()],
                                   "of": "eps = (M_E projected - M_E spherical brute force) / sd(M_E spherical), "
                                         "equal-area annuli about the projection centre"}}
    if accuracy_targets:
        import oracle
        tg = wl.targets.cpu().numpy()
        smp = np.sort(np.random.default_rng(2049).choice(tg, min(accuracy_targets, tg.size), replace=False))
        e1, e2, w = (x.double().cpu().numpy() for x in (cat.e1, cat.e2, cat.w))
        th = wl.theta_ap_arcmin * math.pi / 10800
        ref = oracle.aperture_projected(oracle.pix2vec(wl.nside_out, smp), cat.ra_deg.cpu().numpy(),
                                        cat.dec_deg.cpu().numpy(), e1, e2, w, ra_c, dec_c,
                                        1 if wl.filter == "poly" else 2, th)
        # the plane estimator's normalisation uses the plane area pi theta_ap^2
        ref_n = oracle.finalise_area(ref, math.pi * th * th)
        idx = np.searchsorted(tg, smp)
        it = torch.from_numpy(idx).to(proj["map_e"].device)
        got = {k: v[it].cpu().numpy() for k, v in proj.items()}
        res["accuracy_vs_oracle"] = {
            "targets": int(smp.size), "counts_bit_exact": bool(np.array_equal(got["count"], ref["N"])),
            "rms_rel": {k: float(f"{oracle.rms_rel(got[g].astype(np.float64), ref_n[o]):.3e}")
                        for k, g, o in (("map_e", "map_e", "ME"), ("map_b", "map_b", "MB"), ("var", "var", "VAR"))},
            "tolerance": 1e-4}
    return res


def synth_cap_radius(area_deg2):
    from paper_2609_11181_b300 import synth
    return synth.cap_radius_for_area(area_deg2)


def run_native_galaxy(args, world, rank, peaks_live=None, accuracy_targets=0, projected=False):
    dev = torch.device("cuda", torch.cuda.current_device())
    if peaks_live is None:
        peaks_live = measure_fma_peaks(torch.cuda.current_stream())
    t_gen = time.perf_counter()
    wl = workloads.galaxy_workload(dev, _oracle_centres if accuracy_targets else api.pix2vec,
                                   **GALAXY_WORKLOADS[args.workload])
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    ctx = api.Context(wl.nside_out, wl.theta_ap_arcmin, wl.filter, nside_bin=wl.nside_bin)
    ctx.set_targets(wl.targets)
    cat = wl.cat
    out = ctx._out(None)[0]
    stream = torch.cuda.current_stream()
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        ctx.bin_galaxies(cat.ra_deg, cat.dec_deg, cat.e1, cat.e2, cat.w)
        if evs:
            evs[1].record(stream)
        ctx.map_bruteforce(out)
        if evs:
            evs[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    pairs_step = int(out["members"].long().sum().item())
    clocks = Clocks(torch.cuda.current_device())
    bin_ms = []
    barrier(world)
    torch.cuda.synchronize()
    ctx.timing(True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        step(evs)
        bin_ms.append(evs)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ck = clocks.stop()
    total = t0.elapsed_time(t1) / args.steps
    b_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in bin_ms)
    m_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in bin_ms)
    ms_step = max_over_ranks(total, world)
    value = sum_over_ranks(float(pairs_step), world) / (ms_step * 1e-3) / 1e9
    peak, peak_src = fp32_peak(peaks_live)
    roof, per_kernel = kernel_roofline(
        ctx, {"galaxy": (pairs_step, ALGO_FLOPS_PER_PAIR[wl.filter], BRUTE_EXEC_FLOPS_PER_PAIR[wl.filter],
                         "k_map_galaxy", False)}, args.workload, peak, peak_src)
    phases = {}
    for name in ("bin_keys", "bin_sort", "bin_records", "bin_pixel_sums", "galaxy_band", "galaxy_finalise"):
        nl, ms = ctx.timing_read(name)
        if nl:
            phases[name] = {"launches": nl, "ms_per_launch": round(ms / nl, 4)}
    ctx.timing(False)
    # launches per step: keys (float32 pass, float64 fixes), 4 radix passes of (histogram,
    # scan, scatter), run counts, offsets scan, records, pixel sums; then the three
    # brute-force kernels
    n_gal = cat.n
    ntiles = max(1, -(-n_gal // 4096))
    npix_bin = 12 * wl.nside_bin ** 2
    passes = -(-(npix_bin).bit_length() // 8)
    launches_step = (2 + passes * (2 + scan_launches(256 * ntiles)) + 1 + scan_launches(npix_bin + 1) + 2 + 3)
    res = {"metric": METRIC, "value": round(value, 3), "unit": "Gpair/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload, "desc": wl.desc, "targets": int(wl.targets.numel()),
                      "galaxies": cat.n, "pairs_per_step": pairs_step,
                      "l2": "inputs (2.4 GB catalogue) larger than L2; no flush"},
           "bin_ms": round(b_ms, 3), "map_ms": round(m_ms, 3),
           "roofline": roof, "kernels": per_kernel, "phases": phases,
           "gpu_launches": launches_step * args.steps, "fma_peaks_measured": peaks_live,
           "clocks": ck, "input_gen_s": round(t_gen, 1)}
    if accuracy_targets:
        import oracle
        tg = wl.targets.cpu().numpy()
        smp = np.sort(np.random.default_rng(2048).choice(tg, min(accuracy_targets, tg.size), replace=False))
        e1, e2, w = (x.double().cpu().numpy() for x in (cat.e1, cat.e2, cat.w))
        t_o = time.perf_counter()
        ref = oracle.aperture_galaxies(oracle.pix2vec(wl.nside_out, smp), cat.ra_deg.cpu().numpy(),
                                       cat.dec_deg.cpu().numpy(), e1, e2, w, 1 if wl.filter == "poly" else 2,
                                       wl.theta_ap_arcmin * math.pi / 10800)
        t_o = time.perf_counter() - t_o
        res["accuracy"] = accuracy_vs_oracle(out, tg, smp, ref, wl.theta_ap_arcmin * math.pi / 10800)
        res["accuracy"]["of"] = (f"the timed map at {smp.size} random targets against the float64 oracle's sum "
                                 f"over all {cat.n} galaxies ({t_o:.1f} s on the host)")
    if projected:
        res["projected"] = projected_leg(ctx, wl, cat, out, args.steps, accuracy_targets)
    ctx.close()
    del out, cat, wl
    torch.cuda.empty_cache()
    return res


def run_native_batch(args, world, rank):
    """64 pixel-based maps: 16 binned realisations x 4 apertures, NSIDE 2048."""
    dev = torch.device("cuda", torch.cuda.current_device())
    t_gen = time.perf_counter()
    rng = np.random.default_rng(64)
    ctxs, keep, pairs_total = [], [], 0
    specs = []
    for k in range(16):
        area = float(rng.uniform(500.0, 5000.0))
        dens = float(rng.uniform(10.0, 30.0))                   # gal / arcmin^2
        ra0 = float(rng.uniform(0.0, 360.0))
        dec0 = math.degrees(math.asin(rng.uniform(-0.9, 0.9)))
        mean_count = dens * (4 * math.pi / (12 * 2048 ** 2)) * (180 * 60 / math.pi) ** 2
        wl = workloads.pixel_workload(dev, api.pix2vec, nside=2048, area_deg2=area, mean_count=mean_count,
                                      theta_ap=10.0, filt="schirmer", seed=7000 + k, ra0=ra0, dec0=dec0)
        px = torch.stack([wl.G1, wl.G2, wl.S2, wl.W], dim=1).contiguous()
        keep.append((px, wl.n, wl.targets))
        del wl.G1, wl.G2, wl.S2, wl.W
        for th in (5.0, 10.0, 20.0, 40.0):
            ctx = api.Context(2048, th, "schirmer", nside_bin=2048)
            ctx.set_targets(wl.targets)
            ctx.set_binned_packed(px, wl.n)
            ctxs.append(ctx)
            specs.append(dict(area=round(area), dens=round(dens, 1), theta=th))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.current_stream()
    outs = [c._out(None)[0] for c in ctxs]
    # sequential plain launches
    for _ in range(args.warmup):
        for c, o in zip(ctxs, outs):
            c.map_pixel(o)
    torch.cuda.synchronize()
    pairs_total = sum(int(o["members"].sum().item()) for o in outs)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        for c, o in zip(ctxs, outs):
            c.map_pixel(o)
    t1.record(stream)
    torch.cuda.synchronize()
    seq_ms = t0.elapsed_time(t1) / args.steps
    ref_e = [o["map_e"].clone() for o in outs]
    # one persistent launch in a CUDA graph (autotuned)
    batch = api.Batch(ctxs, outs, autotune=True)
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    barrier(world)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        batch.run()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ck = clocks.stop()
    bat_ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, world)
    same = all(torch.equal(x, o["map_e"]) for x, o in zip(ref_e, outs))
    value = sum_over_ranks(float(pairs_total), world) / (bat_ms * 1e-3) / 1e9
    res = {"metric": METRIC, "value": round(value, 3), "unit": "Gpair/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(bat_ms, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch64", "maps": len(ctxs), "pairs_per_step": pairs_total,
                      "desc": "16 binned realisations (caps 500-5000 deg^2, 10-30 gal/arcmin^2, NSIDE 2048) "
                              "x 4 apertures (5, 10, 20, 40'), Schirmer", "maps_spec": specs[::4],
                      "l2": "inputs (16 GB of binned maps) larger than L2; no flush"},
           "sequential_ms_per_step": round(seq_ms, 3), "batched_speedup": round(seq_ms / bat_ms, 3),
           "batched_equals_sequential": same, "autotune": batch.info(), "clocks": ck, "input_gen_s": round(t_gen, 1)}
    batch.close()
    return res


LEARNED = dict(area_deg2=300.0, n_gal=20_000_000, nside=2048, theta_ap=10.0, filt="schirmer", batch=8192,
               epochs=4, lr=2e-3)


def run_native_learned(args, world, rank):
    """Learned residual correction: maps of seeded 300 deg^2 caps (2e7 galaxies,
    half clumped) at NSIDE 2048, Schirmer 10'; the network is trained on the
    training maps' brute-force minus pixel-based residuals and compared with
    brute force on held-out maps."""
    from paper_2609_11181_b300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    L = LEARNED
    stream = torch.cuda.current_stream()
    ctx = api.Context(L["nside"], L["theta_ap"], L["filt"], nside_bin=L["nside"])
    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
    gen_s, t_bin, t_bf, t_px, t_feat, t_pb, pairs_bf, pairs_px = 0.0, [], [], [], [], [], 0, 0
    train, held = [], []
    n_maps = args.train_maps + args.eval_maps
    for k in range(n_maps):
        rng = np.random.default_rng(9000 + k)
        ra0 = float(rng.uniform(0, 360))
        dec0 = math.degrees(math.asin(rng.uniform(-0.8, 0.8)))
        t0 = time.perf_counter()
        wl = workloads.galaxy_workload(dev, api.pix2vec, n_gal=L["n_gal"], area_deg2=L["area_deg2"],
                                       nside_bin=L["nside"], nside_out=L["nside"], theta_ap=L["theta_ap"],
                                       filt=L["filt"], seed=9000 + k, ra0=ra0, dec0=dec0)
        torch.cuda.synchronize()
        gen_s += time.perf_counter() - t0
        e = [ev() for _ in range(6)]
        ctx.set_targets(wl.targets)
        c = wl.cat
        e[0].record(stream)
        ctx.bin_galaxies(c.ra_deg, c.dec_deg, c.e1, c.e2, c.w)
        e[1].record(stream)
        bf = ctx.map_bruteforce()
        e[2].record(stream)
        px = ctx.map_pixel()
        e[3].record(stream)
        f = ctx.mlp_features(px, bf)
        e[4].record(stream)
        pb = ctx.map_barycentre()
        e[5].record(stream)
        torch.cuda.synchronize()
        t_pb.append(e[4].elapsed_time(e[5]))
        t_bin.append(e[0].elapsed_time(e[1]))
        t_bf.append(e[1].elapsed_time(e[2]))
        t_px.append(e[2].elapsed_time(e[3]))
        t_feat.append(e[3].elapsed_time(e[4]))
        pairs_bf += int(bf["members"].long().sum())
        pairs_px += int(px["members"].long().sum())
        keep = f["valid"].bool()
        d = dict(feat=f["feat"][keep].clone(), target=f["target"][keep].clone(), plain=px["map_e"][keep].clone(),
                 brute=bf["map_e"][keep].clone(), bary=pb["map_e"][keep].clone())
        (train if k < args.train_maps else held).append(d)
        del wl, c, bf, px, f, pb
    feat = torch.cat([d["feat"] for d in train])
    target = torch.cat([d["target"] for d in train])
    net = api.Residual("bf16")
    net.set_params(synth.mlp_init_params(2609))
    net.fit_scaler(feat, target)
    batches = list(synth.minibatches(target.numel(), L["batch"], L["epochs"], seed=2610, device=dev))
    n_steps = len(batches)
    torch.cuda.synchronize()
    tr0, tr1 = ev(), ev()
    tr0.record(stream)
    for k, b in enumerate(batches):
        net.train_step(feat, target, b, L["lr"] if k < 0.75 * n_steps else L["lr"] / 4)
    tr1.record(stream)
    torch.cuda.synchronize()
    train_ms = tr0.elapsed_time(tr1)
    # held-out maps: corrected map (features + inference) against brute force
    t_inf, err_plain, err_corr, eps_plain, eps_corr, err_bary, eps_bary = [], [], [], [], [], [], []
    nfb = torch.zeros(1, dtype=torch.int64, device=dev)
    for d in held:
        a, b = ev(), ev()
        a.record(stream)
        corr = net.infer(d["feat"], d["plain"], n_fallback=nfb)
        b.record(stream)
        torch.cuda.synchronize()
        t_inf.append(a.elapsed_time(b))
        ref = d["brute"].double()
        rms = float(ref.pow(2).mean().sqrt())
        sd = float(ref.std(unbiased=False))
        for m, err, eps in ((d["plain"].double(), err_plain, eps_plain), (corr.double(), err_corr, eps_corr),
                            (d["bary"].double(), err_bary, eps_bary)):
            diff = m - ref
            err.append(float(diff.pow(2).mean().sqrt()) / rms)
            eps.append((float(diff.mean()) / sd, float(diff.std(unbiased=False)) / sd))
    n_held = sum(d["plain"].numel() for d in held)
    ms_px = statistics.mean(t_px)
    ms_learned = ms_px + statistics.mean(t_feat) + statistics.mean(t_inf)
    pairs_px_map = pairs_px / n_maps
    ctx.close()
    return {"metric": METRIC, "value": round(pairs_px_map / (ms_learned * 1e-3) / 1e9, 3), "unit": "Gpair/s",
            "n_gpus": world, "steps": len(held), "warmup": 0, "ms_per_step": round(ms_learned, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
            "data": "synthetic",
            "config": {"workload": "learned", "train_maps": args.train_maps, "eval_maps": args.eval_maps,
                       "desc": f"{L['area_deg2']:.0f} deg^2 caps at seeded centres, {L['n_gal']} galaxies (half "
                               f"clumped, w~U[0.5,1.5]), SIS field, NSIDE {L['nside']} bins and output, "
                               f"{L['filt']} theta_ap={L['theta_ap']}'",
                       "network": "4-64-64-1 SiLU, bf16 weights, f32 accumulation, Adam",
                       "batch": L["batch"], "epochs": L["epochs"], "lr": L["lr"]},
            "forms": {
                "brute_force": {"ms_per_map": round(statistics.mean(t_bf), 3),
                                "bin_ms_per_map": round(statistics.mean(t_bin), 3),
                                "gpair_s": round(pairs_bf / n_maps / (statistics.mean(t_bf) * 1e-3) / 1e9, 3),
                                "rms_err_vs_brute": 0.0},
                "pixel_plain": {"ms_per_map": round(ms_px, 3), "rms_err_vs_brute": round(float(np.mean(err_plain)), 5),
                                "eps_mean": round(float(np.mean([e[0] for e in eps_plain])), 5),
                                "eps_std": round(float(np.mean([e[1] for e in eps_plain])), 5)},
                "pixel_barycentre": {"ms_per_map": round(statistics.mean(t_pb), 3),
                                     "rms_err_vs_brute": round(float(np.mean(err_bary)), 5),
                                     "eps_mean": round(float(np.mean([e[0] for e in eps_bary])), 5),
                                     "eps_std": round(float(np.mean([e[1] for e in eps_bary])), 5),
                                     "note": "first map of a catalogue includes building its records"},
                "pixel_learned": {"ms_per_map": round(ms_learned, 3),
                                  "features_ms": round(statistics.mean(t_feat), 3),
                                  "infer_ms": round(statistics.mean(t_inf), 3),
                                  "rms_err_vs_brute": round(float(np.mean(err_corr)), 5),
                                  "eps_mean": round(float(np.mean([e[0] for e in eps_corr])), 5),
                                  "eps_std": round(float(np.mean([e[1] for e in eps_corr])), 5),
                                  "fallback_pixels": int(nfb.item()), "held_out_pixels": n_held}},
            "training": {"samples": int(target.numel()), "steps": n_steps, "ms": round(train_ms, 1),
                         "samples_per_s": round(n_steps * L["batch"] / (train_ms * 1e-3), 1)},
            "input_gen_s": round(gen_s, 1)}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    # the oracle on this host; one GPU is used only to build the same inputs
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
    import oracle

    def oracle_centres(nside, p):
        return torch.from_numpy(oracle.pix2vec(nside, p.cpu().numpy())).to(p.device)

    wl = workloads.pixel_workload(dev, oracle_centres, **PIXEL_WORKLOADS[args.workload])
    host_G = [x.cpu().numpy() for x in (wl.G1, wl.G2, wl.W, wl.S2, wl.n)]
    times, vals = [], []
    cb = None
    for k in range(args.warmup + args.steps):
        cb, pairs, dt, m = cpu_baseline_pixel(wl, host_G, budget_s=max(1.0, 60.0 / (args.steps + args.warmup)), seed=k)
        if k >= args.warmup:
            times.append(dt)
            vals.append(pairs / dt / 1e9)
    v = statistics.mean(vals)
    return {"metric": METRIC, "value": round(v, 6), "unit": "Gpair/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(times), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "pixel4096", "desc": wl.desc},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": round(v, 6),
                             "unit": "Gpair/s"},
            "e2e": {"value": round(v, 6), "unit": "Gpair/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_forms(args, world, rank, headline: dict) -> dict:
    """The other forms of the metric ("chosen vs plain form"), each at its own
    configuration, timed after the headline in the default run: brute force
    at scale (5e7 galaxies), the batched persistent launch (64 maps), and the
    learned correction with the barycentre form (220 catalogues).  A form
    that fails records its error instead of a result."""
    forms = {"plain_pixel": {"workload": headline["config"]["workload"], "ms_per_map": headline["ms_per_step"],
                             "gpair_s": headline["value"], "accuracy_vs_oracle": headline.get("accuracy")}}
    peaks_live = headline.get("fma_peaks_measured")

    def leg(name, fn):
        t0 = time.perf_counter()
        try:
            forms[name] = fn()
        except Exception as e:                        # noqa: BLE001 -- recorded, the headline stands
            forms[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
        forms[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        torch.cuda.empty_cache()

    def brute():
        a = argparse.Namespace(**vars(args))
        a.workload, a.steps, a.warmup = "brute2048", 3, 3
        r = run_native_galaxy(a, world, rank, peaks_live=peaks_live, accuracy_targets=100, projected=True)
        forms["projected"] = dict(r.pop("projected"), workload="brute2048 (same catalogue and targets)",
                                  form="Cartesian projected estimator projS_pos (Sect. 2.2, 5.2.1)")
        return {"workload": "brute2048", "desc": r["config"]["desc"], "ms_per_step": r["ms_per_step"],
                "bin_ms": r["bin_ms"], "map_ms": r["map_ms"], "gpair_s": r["value"],
                "pairs_per_step": r["config"]["pairs_per_step"], "roofline": r["roofline"],
                "accuracy_vs_oracle": r.get("accuracy"), "clocks": r["clocks"]}

    def batched():
        a = argparse.Namespace(**vars(args))
        a.steps, a.warmup = 3, 3
        r = run_native_batch(a, world, rank)
        return {"workload": "batch64", "desc": r["config"]["desc"], "ms_per_step": r["ms_per_step"],
                "sequential_ms_per_step": r["sequential_ms_per_step"], "batched_speedup": r["batched_speedup"],
                "gpair_s": r["value"], "pairs_per_step": r["config"]["pairs_per_step"],
                "batched_equals_sequential": r["batched_equals_sequential"], "autotune": r["autotune"],
                "clocks": r["clocks"]}

    def learned():
        r = run_native_learned(args, world, rank)
        return {"workload": "learned", "desc": r["config"]["desc"], "forms": r["forms"], "training": r["training"],
                "network": r["config"]["network"]}

    leg("brute_force", brute)
    leg("batched", batched)
    leg("learned", learned)
    return forms


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="pixel4096",
                    choices=sorted(PIXEL_WORKLOADS) + sorted(GALAXY_WORKLOADS) + ["batch64", "learned"])
    ap.add_argument("--train-maps", type=int, default=200)
    ap.add_argument("--eval-maps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the other forms (brute force, batched, learned) after the headline")
    ap.add_argument("--with-projected", action="store_true",
                    help="galaxy workloads: also time the Cartesian projected map on the same catalogue")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        res = run_reference(args, world, rank)
    elif args.workload == "batch64":
        res = run_native_batch(args, world, rank)
    elif args.workload == "learned":
        res = run_native_learned(args, world, rank)
    elif args.workload in GALAXY_WORKLOADS:
        res = run_native_galaxy(args, world, rank, projected=args.with_projected)
    else:
        res = run_native_pixel(args, world, rank)
        if args.workload == "pixel4096" and world == 1 and not args.no_forms:
            res["forms"] = run_forms(args, world, rank, res)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
