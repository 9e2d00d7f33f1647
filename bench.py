"""Throughput of the HELIOS-K opacity hot path on GB300.

One step = one hk_cross_section call over the whole line list at one (T, P):
line strengths, widths, bin geometry, the Voigt sum and the final write
(every step of the path).  Default workload: the 5e8-line water-like list
(log-normal line density over 0-30000 cm^-1), 0.1 cm^-1 grid (3e5 bins),
25 cm^-1 cut, T = 1500 K, P = 1 bar, FP32-compensated arithmetic.

Prints one JSON line.  value = lines/s over all ranks (device time, inputs
resident in HBM); e2e = the same metric with the line list copied from
pinned host memory and sigma copied back inside every timed step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lines/s and Voigt evals/s on 1 GB300 (FP32-comp vs FP64 GPU) at stated σ error"

# Cost model: FP32 flops per (line, bin) pair in each Faddeeva band of the
# FP32-compensated kernel (FMA = 2 flops; reciprocals, exp and sincos counted
# as 1 each): shared x, x^2, r^2 and accumulate = 6; band formulas add 2 (one
# node, r2 >= 1.5e6), 8 (two nodes, r2 >= 2500), 19 (four nodes, r2 >= 64)
# and ~194 for the trapezoid core (r2 < 64).  hk_count_pairs splits the
# four-node range at r2 = 200 (the FP64 kernel's three-node band): both parts
# are four-node work here.  For short lines the kernel evaluates the one-node
# region with the two-node rule (fewer passes per line); the model still counts
# the one-node rule's 8 flops there, so it under-reports rather than inflates.
# ring8: the FP32C short-line batches take the part R8(y) <= r2 < 64 of the
# core with the 8-node Gauss-Hermite rule (four D_j at 4 flops, four numerators
# at 2, their combination over one denominator 11, the reciprocal and scaling
# 3: 6 + 39); hk_count_ring_pairs counts those pairs, which the FP32C rooflines
# take out of the core count.
FLOPS_PER_PAIR = {"gh1": 8, "gh2": 14, "gh3": 25, "gh4": 25, "ring8": 45, "core": 200}
# DRAM bytes per line of one k_gather_f32 launch, from the ncu capture in
# profiles/k_gather_f32_config1-5e7-lines.md (1201.6 MB read + 4.9 MB written for
# 5e7 lines; the line list is read once, so traffic grows with the line
# count).  Set to None when the kernel changes.
GATHER_DRAM_BYTES_PER_LINE = 24.13
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--scale", type=float, default=1.0, help="line-count scale (1 = full)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--adjoint", action="store_true",
                    help="time hk_cross_section_backward over all (T, P) points of the "
                         "workload (config 4) instead of the forward step")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched config-3 launch that follows the headline step")
    ap.add_argument("--table", default=None, metavar="CONFIGS",
                    help="per-configuration throughput table instead of the headline: "
                         "comma-separated config numbers (0-4) and 1x (the options on the "
                         "config-1 list), one JSON line per entry")
    ap.add_argument("--batched", action="store_true",
                    help="time one hk_cross_section_batched launch over every species x "
                         "(T, P) point of the workload (config 3) per step")
    return ap.parse_args()


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def smi_gpu_id(dev):
    """The nvidia-smi id of torch device `dev`: its UUID (GPU-...), which names
    the same physical GPU whatever CUDA_VISIBLE_DEVICES remaps (nvidia-smi -i
    ignores that variable); else the physical index taken from that list."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    idx = dev.index or 0
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if idx < len(ids):
            return ids[idx]
    return str(idx)


def measure_peaks(hk, dev, ms=1000.0):
    """Measured pipe throughputs of this GPU (hk_measure_peak), each with the
    SM clock sampled while it ran: FP32 FMA (scalar, and packed FP32x2), MUFU
    reciprocal and exp2, FP64 FMA (lane operations per second)."""
    out = {}
    for kind, name in [(hk.PEAK_FFMA, "ffma"), (hk.PEAK_FFMA2, "ffma2"), (hk.PEAK_RCP, "mufu_rcp"),
                       (hk.PEAK_EX2, "mufu_ex2"), (hk.PEAK_DFMA, "dfma")]:
        hk.hk_measure_peak(kind, 100.0)
        s = ClockSampler(smi_gpu_id(dev))
        s.start()
        time.sleep(0.25)
        v = hk.hk_measure_peak(kind, ms)
        c = s.stop()
        out[name] = {"ops_per_s": v, "sm_mhz": c.get("sm_mhz"), "reasons": c.get("reasons")}
    return out


def alu_roofline(flops, g_ms, peaks, props, sm_max):
    """Cost-model FLOP/s of the gather against the measured FP32 FMA peak
    (2 flops per FMA), with the nominal unit-count figure beside it."""
    achieved = flops / (g_ms / 1e3) / 1e12
    f = peaks["ffma"]
    peak = 2.0 * f["ops_per_s"] / 1e12
    nominal = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "peak_basis": f"measured FP32 FMA throughput (hk_measure_peak, {f['ops_per_s']:.4g} "
                          f"FMA/s at {f['sm_mhz']} MHz SM clock), x 2 flops",
            "peak_nominal": nominal, "frac_of_nominal": achieved / nominal}


def workload(args):
    from paper_2101_02005_gb300 import synth
    w = synth.config(args.config, scale=args.scale)
    return w


def cpu_sample(w, L, T, P, seconds_target=15.0, nthreads=0, nwin=8):
    """Times the FP64 oracle (as it stands) on nwin seeded windows of the grid:
    the densest, the median and the sparsest 100 cm^-1 log-normal window and
    uniformly drawn positions, each window as many bins wide as takes about
    seconds_target / nwin of oracle time at its own line density (a bin of the
    densest config-1 window already holds ~1e7 pairs), every line within the
    cut of a window included.  Returns pairs/s over all windows, the time, the
    pairs and the windows (lo, hi, oracle sigma, seconds, pairs)."""
    import oracle
    from paper_2101_02005_gb300 import synth
    Q = synth.partition_function
    grid = w.grid.astuple()
    nb = w.grid.nbins
    state = (T, P, float(Q(T)), float(Q(296.0)))
    starts = []
    counts = synth.lognormal_window_counts(L.n, 300, synth.SEED_BASE + w_seed_offset(w)) \
        if L.n >= 300 and nb >= 3000 else None
    if counts is not None:
        order = np.argsort(counts)
        nz = order[counts[order] > 0]
        for widx in (order[-1], order[len(order) // 2], nz[0] if nz.size else order[0]):
            starts.append(int(widx) * (nb // 300) + (nb // 600))
    rng = np.random.default_rng(synth.SEED_BASE + 77)
    while len(starts) < nwin:
        starts.append(int(rng.integers(0, nb)))

    def pairs_in(lo, hi):
        sel = np.searchsorted(L.nu0, [grid[0] + lo * grid[1] - w.cut - grid[1],
                                      grid[0] + hi * grid[1] + w.cut + grid[1]])
        sub = L.subset(slice(int(sel[0]), int(sel[1])))
        rlo, rhi = oracle.line_ranges(sub.nu0, *grid, w.cut)
        n = int(np.clip(np.minimum(rhi, hi - 1) - np.maximum(rlo, lo) + 1, 0, None).sum())
        return sub, n

    # oracle pairs/s from a small probe, to size the windows
    sub, n = pairs_in(starts[1] if len(starts) > 1 else starts[0],
                      (starts[1] if len(starts) > 1 else starts[0]) + 1)
    t0 = time.perf_counter()
    oracle.cross_section(sub.as_oracle(), grid, state, w.cut, starts[1], starts[1] + 1,
                         nthreads=nthreads)
    rate0 = max(n, 1) / max(time.perf_counter() - t0, 1e-4)
    target = rate0 * seconds_target / nwin
    t_used, pairs, wins = 0.0, 0, []
    for st in starts:
        lo = min(max(st, 0), nb - 1)
        _, per_bin = pairs_in(lo, lo + 1)
        width = int(min(2000, max(1, target // max(per_bin, 1))))
        sub, n_pairs = pairs_in(lo, min(nb, lo + width))
        while width > 1 and n_pairs > 1.5 * target:   # a denser neighbour within the cut
            width //= 2
            sub, n_pairs = pairs_in(lo, min(nb, lo + width))
        hi = min(nb, lo + width)
        t0 = time.perf_counter()
        ref = oracle.cross_section(sub.as_oracle(), grid, state, w.cut, lo, hi, nthreads=nthreads)
        dt = time.perf_counter() - t0
        t_used += dt
        pairs += n_pairs
        wins.append((lo, hi, ref, dt, n_pairs))
    return pairs / max(t_used, 1e-9), t_used, pairs, wins


def sample_text(wins, pairs, secs):
    return (f"{len(wins)} seeded windows (densest, median and sparsest 100 cm^-1 log-normal "
            f"window, uniform positions) of " + ", ".join(str(hi - lo) for lo, hi, *_ in wins) +
            f" bins: {pairs} pairs in {secs:.1f} s, pairs/s extrapolated to the whole list")


def max_over_ranks(ms_local, dist, device):
    """The slowest rank's elapsed time (ms): every rank's timed region is
    bracketed by a barrier, and the job takes as long as its slowest rank."""
    if dist is None:
        return float(ms_local)
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_max, steps):
    """Whole-job throughput: the units all ranks processed per second (weak
    scaling: every rank processes units_per_rank per step)."""
    return world * units_per_rank / (ms_max / steps / 1e3)


def w_seed_offset(w):
    return 1 if w.name.startswith("c1") else (2 if w.name.startswith("c2") else 0)


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host cores, same workload
    and metric, each step a bounded window of the grid."""
    import oracle  # noqa: F401
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args)
    L = w.species[0]
    T, P = w.states()[0]
    import oracle as orc
    total_pairs = orc.count_pairs(L.nu0, *w.grid.astuple(), w.cut)
    pairs_per_line = total_pairs / L.n
    cores = os.cpu_count()
    rates = []
    sample = ""
    for s in range(args.warmup + args.steps):
        rate, secs, pairs, wins = cpu_sample(w, L, T, P, seconds_target=4.0)
        if s >= args.warmup:
            rates.append(rate)
        sample = sample_text(wins, pairs, secs) + " (per step)"
    rate = statistics.median(rates)
    value = rate / pairs_per_line
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "lines/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": L.n / value * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "lines": L.n, "bins": w.grid.nbins,
                       "pairs": total_pairs},
            "e2e": {"value": value, "unit": "lines/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": value, "unit": "lines/s", "cores": cores,
                             "kind": "oracle", "sample": sample,
                             "note": "extrapolated from pairs/s over the whole list"}}
    print(json.dumps(line), flush=True)


def run_adjoint(args, w, hk, synth, dev):
    """The adjoint of the workload's (T, P) points (config 4: dL/dT, dL/dP and
    per-line dL/dS_ref, dL/dgamma_ref from an N(0, 1) upstream gradient)."""
    import torch
    Q = synth.partition_function
    L = w.species[0]
    pts = w.states()
    D = hk.DeviceLines.from_host(L)
    grid = hk.make_grid(*w.grid.astuple())
    opts = hk.make_opts(float(Q(296.0)), w.cut)
    states = [hk.make_state(t, p, float(Q(t)), float(synth.dlnQ_dT(t))) for t, p in pts]
    g = torch.from_numpy(synth.upstream_grad(len(pts), w.grid.nbins,
                                             synth.SEED_BASE + args.config)).to(dev)
    pairs = sum(hk.hk_count_pairs(D, grid, s, opts)[0] for s in states)
    for _ in range(args.warmup):
        hk.hk_cross_section_backward(D, grid, states, opts, g)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        hk.hk_cross_section_backward(D, grid, states, opts, g)
    e1.record()
    torch.cuda.synchronize()
    hk.hk_sync_status()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"metric": "adjoint line-points/s", "value": L.n * len(pts) / (ms / 1e3),
                      "unit": "line-points/s", "ms_per_step": ms, "steps": args.steps,
                      "warmup": args.warmup, "derivative_evals_per_s": pairs / (ms / 1e3),
                      "higher_is_better": True,
                      "config": {"workload": w.name, "lines": L.n, "points": len(pts),
                                 "pairs_per_step": pairs}}), flush=True)


def run_batched(args, w, hk, synth, dev):
    """Prints the batched measurement of the workload as its own JSON line."""
    peaks = measure_peaks(hk, dev)
    print(json.dumps(batched_measure(w, hk, synth, dev, args.steps, args.warmup, peaks)),
          flush=True)


def batched_measure(w, hk, synth, dev, steps, warmup, peaks):
    """One step = one persistent batched launch over every species at every
    (T, P) point of the workload (config 3: 4 species x 200 points, sigma in
    FP64, 12.8 GB); lines per work item from the library's autotuner on the
    largest species at the middle point.  Pair and band counts (for the cost
    model) come from hk_count_pairs, outside the timed region."""
    import torch
    Q = synth.partition_function
    species = [hk.DeviceLines.from_host(s) for s in w.species]
    grid = hk.make_grid(*w.grid.astuple())
    opts = hk.make_opts(float(Q(296.0)), w.cut, hk.HK_FP32C, flags=hk.HK_SIGMA_F64)
    pts = w.states()
    states = [hk.make_state(t, p, float(Q(t))) for t, p in pts]
    counts = [0] * 7
    for s in species:
        for st in states:
            c = hk.hk_count_pairs(s, grid, st, opts) + [hk.hk_count_ring_pairs(s, grid, st, opts)]
            counts = [a + b for a, b in zip(counts, c)]
    bands = dict(zip(["gh1", "gh2", "gh3", "gh4", "core", "ring8"], counts[1:]))
    bands["core"] -= bands["ring8"]
    flops_step = sum(FLOPS_PER_PAIR[b] * n for b, n in bands.items())
    big = max(range(len(species)), key=lambda i: species[i].n)
    hk.hk_autotune(species[big], grid, states[len(states) // 2], opts)
    lmax, tile_bins = hk.hk_tuning_full(hk.HK_FP32C)
    need = hk.hk_workspace_size(0, species, len(states), grid, opts)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    out = torch.empty((len(species), len(states), w.grid.nbins), dtype=torch.float64, device=dev)

    def step():
        hk.hk_cross_section_batched(species, states, grid, opts, out, ws)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    hk.hk_sync_status()
    sampler = ClockSampler(smi_gpu_id(dev))
    sampler.start()
    time.sleep(0.3)
    hk.hk_profile(1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    gather_ms, launches = hk.hk_profile(0)
    clocks = sampler.stop()
    hk.hk_sync_status()
    ms = e0.elapsed_time(e1) / steps
    g_ms = gather_ms / max(launches, 1)
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(load_peaks().get("sm_max_mhz", 2070.0))
    roof = alu_roofline(flops_step, g_ms, peaks, props, sm_max)
    roof.update({"kernel": "k_gather_f32", "gather_ms_per_launch": g_ms,
                 "cost_model": FLOPS_PER_PAIR})
    line_points = sum(s.n for s in species) * len(states)
    out_ = {"metric": "batched line-points/s", "value": line_points / (ms / 1e3),
            "unit": "line-points/s", "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "voigt_evals_per_s": counts[0] / (ms / 1e3),
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "roofline": roof, "clocks": clocks,
            "config": {"workload": w.name, "species_lines": [s.n for s in species],
                       "points": len(states), "pairs_per_step": counts[0],
                       "band_pairs": bands, "lmax_autotuned": lmax,
                       "tile_bins_autotuned": tile_bins,
                       "sigma_out": "f64", "call": "hk_cross_section_batched"}}
    del out, ws, species
    torch.cuda.empty_cache()
    return out_


def run_table(args, hk, synth, dev):
    """Throughput of every configuration (0-4) at its full size, one JSON line
    per entry: the FP32-compensated path (device-resident lines, sigma in FP64)
    and the plain FP64 GPU form (on an every-k-th-line sample where the full
    list would take minutes; a line's work does not depend on the density),
    each with its own autotuned lines per work item (FP64: tuned on at most
    5e6 lines of the list), SM clocks sampled during the timed launches, and
    the oracle's pairs/s on seeded windows (config 0: the whole array).  The
    per-configuration errors against the oracle come from the full-size GPU
    tests, which record them."""
    import torch
    Q = synth.partition_function
    qref = float(Q(296.0))
    keys = [c.strip() for c in args.table.split(",") if c.strip()]
    only = [int(c) for c in keys if c.isdigit()]

    def emit(d):
        print(json.dumps(d), flush=True)

    def timed(fn, reps, warm=2):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        smp = ClockSampler(smi_gpu_id(dev))
        smp.start()
        time.sleep(0.25)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        c = smp.stop()
        hk.hk_sync_status()
        return e0.elapsed_time(e1) / reps, c

    def single(tag, L, grid_t, T, P, cut, prec, reps, every=None):
        Ls = L if every is None else L.subset(slice(0, None, every))
        D = hk.DeviceLines.from_host(Ls)
        grid = hk.make_grid(*grid_t)
        st = hk.make_state(T, P, float(Q(T)))
        op = hk.make_opts(qref, cut, prec, flags=hk.HK_SIGMA_F64 if prec == hk.HK_FP32C else 0)
        out = torch.empty(grid_t[2], dtype=torch.float64, device=dev)
        if prec == hk.HK_FP64 and Ls.n > 5_000_000:
            Dt = hk.DeviceLines.from_host(Ls.subset(slice(0, None, -(-Ls.n // 5_000_000))))
            hk.hk_autotune(Dt, grid, st, op)
            del Dt
        else:
            hk.hk_autotune(D, grid, st, op)
        pairs = hk.hk_count_pairs(D, grid, st, op)[0]
        ms, c = timed(lambda: hk.hk_cross_section(D, grid, st, op, out), reps)
        emit({"table": tag, "precision": "fp64" if prec else "fp32c", "lines": Ls.n,
              "sample": f"every {every}th line" if every else "all lines", "ms": ms,
              "lines_per_s": Ls.n / (ms / 1e3), "evals_per_s": pairs / (ms / 1e3),
              "pairs": pairs, "tuning": hk.hk_tuning_full(prec),
              "sm_mhz": c.get("sm_mhz"), "reasons": c.get("reasons")})
        del D, out
        torch.cuda.empty_cache()

    def oracle_rate(tag, w, L, T, P, secs=8.0):
        rate, t_used, pairs, wins = cpu_sample(w, L, T, P, seconds_target=secs)
        emit({"table": tag, "oracle_pairs_per_s": rate, "cores": os.cpu_count(),
              "pairs": pairs, "seconds": t_used, "sample": sample_text(wins, pairs, t_used)})

    if 0 in only:
        w = synth.config(0)
        L = w.species[0]
        T, P = w.states()[0]
        for prec in (hk.HK_FP32C, hk.HK_FP64):
            single("c0", L, w.grid.astuple(), T, P, w.cut, prec, 20)
        import oracle
        t0 = time.perf_counter()
        oracle.cross_section(L.as_oracle(), w.grid.astuple(), (T, P, float(Q(T)), qref), w.cut)
        dt = time.perf_counter() - t0
        emit({"table": "c0 oracle (whole array)", "seconds": dt, "cores": os.cpu_count(),
              "oracle_pairs_per_s": oracle.count_pairs(L.nu0, *w.grid.astuple(), w.cut) / dt})
    if 1 in only:
        w = synth.config(1)
        L = w.species[0]
        T, P = w.states()[0]
        single("c1", L, w.grid.astuple(), T, P, w.cut, hk.HK_FP32C, 5)
        single("c1", L, w.grid.astuple(), T, P, w.cut, hk.HK_FP64, 1, every=10)
        oracle_rate("c1 oracle", w, L, T, P)
        del w, L
    if "1x" in keys:
        # the options of Sect. 2.1 and 2.4.3 on the config-1 list, one call each
        # (autotuned per option set): plinth, per-line cuts, other profiles
        w = synth.config(1)
        L = w.species[0]
        T, P = w.states()[0]
        D = hk.DeviceLines.from_host(L)
        grid = hk.make_grid(*w.grid.astuple())
        st = hk.make_state(T, P, float(Q(T)))
        out = torch.empty(w.grid.nbins, dtype=torch.float64, device=dev)
        modes = [("Voigt, cut 25", {}),
                 ("Voigt, plinth removed", {"flags": hk.HK_REMOVE_PLINTH}),
                 ("Voigt, cut 1000 Doppler widths", {"cut_mode": hk.HK_CUT_DOPPLER, "cut": 1000.0}),
                 ("Voigt, cut 500 Lorentz widths", {"cut_mode": hk.HK_CUT_LORENTZ, "cut": 500.0}),
                 ("Lorentzian, cut 25", {"profile": hk.HK_PROFILE_LORENTZ}),
                 ("Doppler, cut 25", {"profile": hk.HK_PROFILE_DOPPLER}),
                 ("binned Gaussian, cut 25", {"profile": hk.HK_PROFILE_BINNED_GAUSS})]
        for name, kw in modes:
            kw = dict(kw)
            cut = kw.pop("cut", w.cut)
            flags = kw.pop("flags", 0) | hk.HK_SIGMA_F64
            op = hk.make_opts(qref, cut, hk.HK_FP32C, flags=flags, **kw)
            hk.hk_autotune(D, grid, st, op)
            pairs = hk.hk_count_pairs(D, grid, st, op)[0]
            ms, c = timed(lambda: hk.hk_cross_section(D, grid, st, op, out), 3)
            emit({"table": f"c1 option: {name}", "precision": "fp32c", "lines": L.n, "ms": ms,
                  "lines_per_s": L.n / (ms / 1e3), "evals_per_s": pairs / (ms / 1e3),
                  "pairs": pairs, "tuning": hk.hk_tuning_full(hk.HK_FP32C),
                  "sm_mhz": c.get("sm_mhz"), "reasons": c.get("reasons")})
        del D, out, w, L
        torch.cuda.empty_cache()
    if 2 in only:
        w = synth.config(2)
        L = w.species[0]
        T, P = w.states()[0]
        single("c2 molecules", L, w.grid.astuple(), T, P, w.cut, hk.HK_FP32C, 3)
        single("c2 molecules", L, w.grid.astuple(), T, P, w.cut, hk.HK_FP64, 1, every=100)
        oracle_rate("c2 molecules oracle", w, L, T, P)
        A = w.extra["atoms"]
        ag = w.extra["atom_grid"].astuple()
        single("c2 atoms", A, ag, T, P, 0.0, hk.HK_FP32C, 3)
        single("c2 atoms", A, ag, T, P, 0.0, hk.HK_FP64, 1, every=100)
        del w, L, A
    if 3 in only:
        w = synth.config(3)
        T, P = w.T[10], w.P[5]
        for s_, L in enumerate(w.species):
            single(f"c3 species {s_} one point", L, w.grid.astuple(), T, P, w.cut,
                   hk.HK_FP64, 1, every=10 if L.n > 1e6 else None)
        oracle_rate("c3 species 3 oracle (one point)", w, w.species[3], T, P)
        del w
    if 4 in only:
        w = synth.config(4)
        L = w.species[0]
        pts = w.states()
        D = hk.DeviceLines.from_host(L)
        grid = hk.make_grid(*w.grid.astuple())
        states = [hk.make_state(t, p, float(Q(t)), float(synth.dlnQ_dT(t))) for t, p in pts]
        op = hk.make_opts(qref, w.cut, hk.HK_FP32C, flags=hk.HK_SIGMA_F64)
        hk.hk_autotune(D, grid, states[len(states) // 2], op)
        out = torch.empty((1, len(pts), w.grid.nbins), dtype=torch.float64, device=dev)
        ws = torch.empty(hk.hk_workspace_size(0, [D], len(pts), grid, op), dtype=torch.uint8,
                         device=dev)
        pairs = sum(hk.hk_count_pairs(D, grid, st_, op)[0] for st_ in states)
        ms, c = timed(lambda: hk.hk_cross_section_batched([D], states, grid, op, out, ws), 3)
        emit({"table": "c4 forward (16 points, batched)", "precision": "fp32c", "ms": ms,
              "lines_per_s": L.n * len(pts) / (ms / 1e3), "evals_per_s": pairs / (ms / 1e3),
              "sm_mhz": c.get("sm_mhz"), "reasons": c.get("reasons")})
        g = torch.from_numpy(synth.upstream_grad(len(pts), w.grid.nbins,
                                                 synth.SEED_BASE + 4)).to(dev)
        ms, c = timed(lambda: hk.hk_cross_section_backward(D, grid, states,
                                                           hk.make_opts(qref, w.cut), g), 3)
        emit({"table": "c4 adjoint (16 points)", "ms": ms,
              "line_points_per_s": L.n * len(pts) / (ms / 1e3),
              "derivative_evals_per_s": pairs / (ms / 1e3), "sm_mhz": c.get("sm_mhz"),
              "reasons": c.get("reasons")})
        del D, out, ws, g
        torch.cuda.empty_cache()
        T, P = pts[5]
        single("c4 one point", L, w.grid.astuple(), T, P, w.cut, hk.HK_FP64, 1)
        oracle_rate("c4 oracle (point 5)", w, L, T, P)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2101_02005_gb300 import build as pbuild
    pbuild.build()
    from paper_2101_02005_gb300 import hk, synth

    if args.table is not None:
        run_table(args, hk, synth, dev)
        return
    peaks_m = measure_peaks(hk, dev)
    t_gen = time.perf_counter()
    w = workload(args)
    L = w.species[0]
    T, P = w.states()[0]
    Q = synth.partition_function
    t_gen = time.perf_counter() - t_gen
    if args.adjoint:
        run_adjoint(args, w, hk, synth, dev)
        return
    if args.batched:
        print(json.dumps(batched_measure(w, hk, synth, dev, args.steps, args.warmup, peaks_m)),
              flush=True)
        return

    # line list resident in HBM; pinned host copies for the end-to-end timing
    host = {k: torch.from_numpy(getattr(L, k)) for k in ("nu0", "S_ref", "E_low", "gamma_ref", "n_T")}
    D = hk.DeviceLines(*(host[k].to(dev) for k in ("nu0", "S_ref", "E_low", "gamma_ref", "n_T")),
                       L.mass_amu, s_mode=L.s_mode, sorted=L.sorted)
    grid = hk.make_grid(*w.grid.astuple())
    state = hk.make_state(T, P, float(Q(T)), float(synth.dlnQ_dT(T)))
    opts = hk.make_opts(float(Q(296.0)), w.cut, hk.HK_FP32C, flags=hk.HK_SIGMA_F64)
    sigma = torch.empty(w.grid.nbins, dtype=torch.float64, device=dev)
    counts = hk.hk_count_pairs(D, grid, state, opts)
    pairs = counts[0]
    bands = dict(zip(["gh1", "gh2", "gh3", "gh4", "core"], counts[1:]))
    bands["ring8"] = hk.hk_count_ring_pairs(D, grid, state, opts)
    bands["core"] -= bands["ring8"]
    flops_step = sum(FLOPS_PER_PAIR[b] * n for b, n in bands.items())
    stream = torch.cuda.current_stream()

    def step():
        hk.hk_cross_section(D, grid, state, opts, sigma)

    # the library's autotuner picks the lines per work item once (untimed)
    t_tune = time.perf_counter()
    hk.hk_autotune(D, grid, state, opts)
    t_tune = time.perf_counter() - t_tune
    lmax, tile_bins = hk.hk_tuning_full(hk.HK_FP32C)

    for _ in range(args.warmup):
        step()
    hk.hk_sync_status()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(smi_gpu_id(dev))
    barrier()
    sampler.start()
    time.sleep(0.3)
    hk.hk_profile(1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    gather_ms, gather_launches = hk.hk_profile(0)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    hk.hk_sync_status()
    ms_max = max_over_ranks(ms, dist, dev)
    ms_step = ms_max / args.steps
    value = job_rate(L.n, world, ms_max, args.steps)

    # roofline of the dominant kernel (the Voigt gather), live CUDA-event time,
    # against the FP32 FMA peak measured on this GPU at the start of the run
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(load_peaks().get("sm_max_mhz", 2070.0))
    g_ms = gather_ms / max(gather_launches, 1)
    traffic = (GATHER_DRAM_BYTES_PER_LINE * L.n
               if GATHER_DRAM_BYTES_PER_LINE and args.config == 1 else None)
    roofline = alu_roofline(flops_step, g_ms, peaks_m, props, sm_max)
    roofline.update({
        "kernel": ("k_gather_f32<0> (batched short-line sweeps)"
                   if 2 * w.cut / w.grid.dnu + 1 < 1024 else "k_gather_f32<1> (peeled sweeps)"),
        "traffic": traffic,
        "traffic_basis": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one 5e7-line "
                          "launch of this kernel (profiles/k_gather_f32_config1-5e7-lines.md), "
                          "24.1 B per line, scaled by the line count" if traffic else None),
        "algorithmic_bytes": 24 * L.n, "gather_ms_per_launch": g_ms,
        "gather_share_of_step": g_ms / ms_step if ms_step else None,
        "flops_per_step": flops_step, "cost_model": FLOPS_PER_PAIR,
        "measured_peaks": peaks_m})

    # end to end through the host-buffer entry point: the line list in pinned
    # host memory is streamed to the GPU in blocks whose copies overlap the
    # sums, sigma comes back to pinned host memory, all inside the timed region
    e2e = None
    if not args.no_e2e:
        H = hk.HostLines(*(host[k].pin_memory() for k in ("nu0", "S_ref", "E_low", "gamma_ref",
                                                           "n_T")),
                         L.mass_amu, s_mode=L.s_mode, sorted=L.sorted)
        out_h = torch.empty(w.grid.nbins, dtype=torch.float64).pin_memory()
        h2d = sum(getattr(H, k).numel() * getattr(H, k).element_size()
                  for k in ("nu0", "S_ref", "E_low", "gamma_ref", "n_T"))
        d2h = out_h.numel() * out_h.element_size()

        def e2e_step():
            hk.hk_cross_section_host(H, grid, state, opts, out_h, stream=stream)

        e2e_step()
        barrier()
        esampler = ClockSampler(smi_gpu_id(dev))
        esampler.start()
        time.sleep(0.3)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        f1.record(stream)
        barrier()
        eclocks = esampler.stop()
        ems = max_over_ranks(f0.elapsed_time(f1), dist, dev)
        e2e = {"value": job_rate(L.n, world, ems, args.steps), "unit": "lines/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": ems / args.steps, "call": "hk_cross_section_host",
               "block_lines": 1 << 26, "clocks": eclocks}
        del H

    # the plain FP64 GPU form on every 10th line (per-line work is the same
    # for every line: the cut admits 2 cut/dnu + 1 bins whatever the density)
    fp64 = None
    if not args.no_fp64:
        sub = slice(0, None, 10)
        D64 = hk.DeviceLines(D.nu0[sub].contiguous(), D.S_ref[sub].contiguous(),
                             D.E_low[sub].contiguous(), D.gamma_ref[sub].contiguous(),
                             D.n_T[sub].contiguous(), L.mass_amu)
        o64 = hk.make_opts(float(Q(296.0)), w.cut, hk.HK_FP64)
        s64 = torch.empty(w.grid.nbins, dtype=torch.float64, device=dev)
        # the FP64 form's own lines per work item, from the autotuner on every
        # 10th line of the sample (untimed)
        sub10 = slice(0, None, 10)
        Dt = hk.DeviceLines(D64.nu0[sub10].contiguous(), D64.S_ref[sub10].contiguous(),
                            D64.E_low[sub10].contiguous(), D64.gamma_ref[sub10].contiguous(),
                            D64.n_T[sub10].contiguous(), L.mass_amu)
        hk.hk_autotune(Dt, grid, state, o64)
        del Dt
        lmax64 = hk.hk_tuning_full(hk.HK_FP64)[0]
        hk.hk_cross_section(D64, grid, state, o64, s64)
        torch.cuda.synchronize()
        hk.hk_profile(1)
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        hk.hk_cross_section(D64, grid, state, o64, s64)
        g1.record(stream)
        torch.cuda.synchronize()
        g64_ms, _ = hk.hk_profile(0)
        f64ms = g0.elapsed_time(g1)
        c64 = hk.hk_count_pairs(D64, grid, state, o64)
        flops64 = sum(FLOPS_PER_PAIR[b] * n for b, n in
                      zip(["gh1", "gh2", "gh3", "gh4", "core"], c64[1:]))
        achieved64 = flops64 / (g64_ms / 1e3) / 1e12
        peak64 = 2.0 * peaks_m["dfma"]["ops_per_s"] / 1e12
        fp64 = {"value": D64.n / (f64ms / 1e3), "unit": "lines/s", "lmax_autotuned": lmax64,
                "voigt_evals_per_s": c64[0] / (f64ms / 1e3), "ms": f64ms,
                "sample": "every 10th line of the list, one step; every line admits the same "
                          "2 cut/dnu + 1 bins whatever the density, so the whole list takes "
                          "10x as long (%.1f s)" % (10 * f64ms / 1e3),
                "fp32c_speedup": (D64.n / (f64ms / 1e3)) and value / (D64.n / (f64ms / 1e3)),
                "roofline": {"bound": "fp64", "kernel": "k_gather<double, 2>",
                             "achieved": achieved64, "peak": peak64, "unit": "TFLOP/s",
                             "frac": achieved64 / peak64, "gather_ms": g64_ms,
                             "peak_basis": "measured FP64 FMA throughput (hk_measure_peak) x 2",
                             "cost_model": "the FP32C gather's flops per pair and band"}}
        del D64, s64

    # the batched opacity table (config 3: 4 species x 200 (T, P) points in one
    # persistent launch, FP32C), reported beside the headline; its line list
    # replaces the headline's on the device
    batched = None
    if not args.no_batched and rank == 0 and args.config == 1 and args.scale == 1.0:
        got_sigma = sigma.cpu().numpy()
        del D, sigma
        torch.cuda.empty_cache()
        w3 = synth.config(3)
        batched = batched_measure(w3, hk, synth, dev, 1, 1, peaks_m)
        del w3
    else:
        got_sigma = None

    # CPU baseline (oracle as it stands, host cores) on a bounded sample, which
    # doubles as a parity check of this run's sigma on the same bins
    cpu = None
    parity = None
    if not args.no_cpu and rank == 0:
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from parity import sampled_errors
        from parity import sigma_errors as sigma_errors_window
        rate, secs, cpairs, wins = cpu_sample(w, L, T, P, seconds_target=15.0)
        pairs_per_line = pairs / L.n
        cpu = {"value": rate / pairs_per_line, "unit": "lines/s", "cores": os.cpu_count(),
               "kind": "oracle", "voigt_evals_per_s": rate,
               "sample": sample_text(wins, cpairs, secs), "extrapolated": True}
        got = got_sigma if got_sigma is not None else sigma.cpu().numpy()
        # the bar's mask: bins above 1e-10 of the whole array's maximum (FP32C
        # flushes contributions ~2^-126 below the largest line peak, so bins
        # far below the array's maximum may read 0 -- outside the mask)
        gmax = float(np.max(got))
        errs = [sigma_errors_window(got[lo:hi], ref, ref_max=gmax) for lo, hi, ref, _, _ in wins]
        # and a seeded sample of bins over the whole array (uniform, above the
        # mask, the maximum), the oracle one bin at a time
        es = sampled_errors(got, L, w.grid.astuple(), (T, P, float(Q(T)), float(Q(296.0))),
                            w.cut, 11)
        parity = {"windows": {"rel_l1": max(e["l1"] for e in errs),
                              "max_bin_rel": max(e["max_bin"] for e in errs),
                              "bins": int(sum(hi - lo for lo, hi, _, _, _ in wins)),
                              "bins_above_mask": int(sum(e["n_mask"] for e in errs))},
                  "sampled_bins": {"rel_l1": es["l1"], "max_bin_rel": es["max_bin"],
                                   "bins": es["n"], "bins_above_mask": es["n_mask"]},
                  "bar": "rel L1 <= 1e-5, per bin <= 1e-4 over bins above 1e-10 of the "
                         "array's maximum"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "lines/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "lines_per_gpu": L.n, "bins": w.grid.nbins,
                           "voigt_pairs_per_step": pairs, "precision": "FP32-compensated",
                           "sigma_out": "f64",
                           "l2": "inputs (24 B/line, %.1f GB) larger than L2" % (24 * L.n / 1e9),
                           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                           "band_pairs": bands, "generation_s": round(t_gen, 1),
                           "lmax_autotuned": lmax, "tile_bins_autotuned": tile_bins,
                           "autotune_s": round(t_tune, 2)},
                "voigt_evals_per_s": world * pairs / (ms_step / 1e3),
                # per hk_cross_section: descriptor upload, scale prepass, tile
                # ranges, scan, gather, finalize (see the launch list profile)
                "gpu_launches": 6 * args.steps,
                "roofline": roofline, "clocks": clocks, "e2e": e2e, "fp64_gpu": fp64,
                "cpu_baseline": cpu, "parity_sample": parity, "batched_c3": batched}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
