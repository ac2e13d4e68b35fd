#!/usr/bin/env python
"""Benchmark of the checkerboard SU(3) gauge sweep on GB300.

Workload: SU(3) Wilson action on a 64^3 x 16 lattice (4.2M sites), beta 6.2,
constant lambda3 background field with flux quantum n = 1, hot start, links
stored in FP32 (12 reals per link, third row rebuilt).  One step = one working
sweep: 1 Cabibbo-Marinari heat-bath pass + 4 overrelaxation passes + FP64
reunitarization + plaquette / Polyakov-loop measurement (FP64 sums).  The
links (805 MB) are larger than L2 (129 MB), so no L2 flush is needed.

Metric: link updates per second (one heat-bath or one overrelaxation update of
one link = one update).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica (its own seed)
and rank 0 reports the units of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "link updates/sec and HBM GB/s (% of peak), FP32-batched vs FP64 plain, |dP|<=1e-6"
UNIT = "link updates/s"
# link bytes per storage; algorithmic traffic per link update is 9 link
# transfers (3V links of the other directions, V/2 opposite-parity links of the
# same direction, V/2 read + V/2 written, for V/2 updates per phase).
LINK_BYTES = {(3, 1): 48, (3, 0): 144, (2, 1): 16, (2, 0): 32}
TRANSFERS_PER_UPDATE = 9
# FP64 flops of one SU(3) overrelaxation update in the FP64 kernel (FMA = 2):
# staple 12 full 3x3 complex products (324 complex multiply-adds), W = U A
# (27), the three subgroup rotations of U and the first two of W (60), at 8
# flops each = 3,288, plus ~150 for the projections, norms and quaternion
# squares.  The peak it is held to is measured in the run (qcd_probe_fp64_rate:
# FP64 FMA chains filling every SM, CUDA events); the nominal 1.25 TFLOP/s of
# GB300 (152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz) is the fallback.
FP64_OR_FLOPS = 3438
FP64_PEAK_TFLOPS_NOMINAL = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64-plain and batched-scan side measurements")
    ap.add_argument("--batch-only", action="store_true",
                    help="time only the batched 64-lattice scan (--steps sweeps in one launch)")
    ap.add_argument("--batch-copies", type=int, default=1,
                    help="with --batch-only: repeat the scan's lattice list (8 copies outgrow L2)")
    ap.add_argument("--Ns", type=int, default=None, help="override the spatial extent (small profiling cases)")
    ap.add_argument("--Nt", type=int, default=None, help="override the time extent (small profiling cases)")
    ap.add_argument("--storage", choices=["fp32", "fp64"], default="fp32",
                    help="link storage of the timed lattice (fp64: FP64 18-real, for profiling the FP64 kernels)")
    return ap.parse_args()


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Source files that define the SU(3) FP32 phase kernels (the dominant kernel).
PHASE_KERNEL_SOURCES = ("qcd_device.cuh", "qcd_internal.h", "qcd_kernels.cuh", "qcd_su3c.cuh", "su3_f32.cu")


def kernel_source_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1310_7087_gb300", "csrc")
    for name in PHASE_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_kind, workload):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel sources and on this
    workload; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel_kind)
    if not e or e.get("source_sha") != kernel_source_sha() or e.get("config") != workload:
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed
    region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_index: int):
        self.samples = []
        self.window = None
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.time(), parts))

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()
        time.sleep(0.25)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        inside = [p for t, p in self.samples if self.t0 - 0.1 <= t <= self.t1 + 0.1]
        if not inside:
            inside = [p for _, p in self.samples]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for p in inside if num(p[1]) is not None]
        mx = [num(p[2]) for p in inside if num(p[2]) is not None]
        reasons = sorted({n for p in inside for n, v in zip(self.NAMES, p[4:8]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


def cpu_baseline_oracle(w):
    """The oracle as it stands, on all host cores, on a bounded sample of the
    same workload: one heat-bath pass, one overrelaxation pass, one
    reunitarization and one measurement of the full lattice, combined with the
    sweep's 1 : 4 pass mix."""
    import oracle
    oracle.build()
    L = oracle.OracleLattice(w.group, w.Ns, w.Nt, w.beta, w.flux, w.nhit, 0)
    L.hot_start(w.seed)
    t = {}
    t0 = time.perf_counter()
    for p in range(2):
        for mu in range(4):
            L.phase(oracle.HEATBATH, p, mu, w.seed)
    t["hb"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    for p in range(2):
        for mu in range(4):
            L.phase(oracle.OVERRELAX, p, mu, w.seed)
    t["or"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    L.reunitarize()
    t["re"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    L.measure()
    t["me"] = time.perf_counter() - t0
    L.close()
    sweep_s = t["hb"] + w.n_or * t["or"] + t["re"] + t["me"]
    lu = (1 + w.n_or) * 4 * w.volume
    return {"value": lu / sweep_s, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": "one HB pass, one OR pass, one reunitarization and one measurement of the full "
                      "%s lattice (%.1f s of CPU work), combined as 1 HB + %d OR per sweep"
                      % (w.name, sum(t.values()), w.n_or),
            "seconds": {k: round(v, 3) for k, v in t.items()},
            "hb_lu_per_s": 4 * w.volume / t["hb"], "or_lu_per_s": 4 * w.volume / t["or"],
            "sweeps_per_s": 1.0 / sweep_s, "cpu": cpu_model(), "plan": oracle_plan(oracle)}


def cpu_model():
    import platform
    name = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    name = "%s (%s)" % (platform.machine(), line.split(":", 1)[1].strip())
                    break
    except OSError:
        pass
    return {"model": name, "nproc": os.cpu_count()}


def oracle_plan(oracle):
    """Oracle timings on the small configurations (link updates/s, all host
    cores unless noted): SU(2) 4^3x4 cold, 100 x (1 HB + 1 OR); SU(3) 16^3x4,
    1 HB + 4 OR + reunitarization (also single-threaded); SU(2) and SU(3) 8^4,
    sweeps of 1 HB + reunitarization without measurements, as in the paper's
    8^4 comparison; SU(3) 32^3x8 two sweeps of 1 HB + 4 OR (a rate, so it
    stands for a longer run)."""
    def run(N, Ns, Nt, beta, n_hb_sweeps, n_or, seed, cold=False, threads=None):
        n0 = oracle.get_threads()
        if threads:
            oracle.set_threads(threads)
        try:
            L = oracle.OracleLattice(N, Ns, Nt, beta, 0, 10, 0)
            if not cold:
                L.hot_start(seed)
            t0 = time.perf_counter()
            L.sweep(n_hb_sweeps, n_or, seed)
            dt = time.perf_counter() - t0
            L.close()
        finally:
            oracle.set_threads(n0)
        lu = n_hb_sweeps * (1 + n_or) * 4 * Ns ** 3 * Nt
        return {"lu_per_s": lu / dt, "seconds": round(dt, 3), "sweeps": n_hb_sweeps}
    return {"su2_4^3x4_cold_100x(1HB+1OR)": run(2, 4, 4, 2.3, 100, 1, 1, cold=True),
            "su3_16^3x4_1HB+4OR": run(3, 16, 4, 5.7, 1, 4, 7),
            "su3_16^3x4_1HB+4OR_1thread": run(3, 16, 4, 5.7, 1, 4, 7, threads=1),
            "su2_8^4_1HB": run(2, 8, 8, 2.3, 10, 0, 3),
            "su3_8^4_1HB": run(3, 8, 8, 5.7, 4, 0, 3),
            "su3_32^3x8_2x(1HB+4OR)": run(3, 32, 8, 6.0, 2, 4, 5)}


def run_reference(args, w):
    """Reference arm: the FP64 CPU oracle timed on the host cores."""
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    L = oracle.OracleLattice(w.group, w.Ns, w.Nt, w.beta, w.flux, w.nhit, 0)
    L.hot_start(w.seed)
    Vh = w.volume // 2
    schedule = []
    for i in range(1 + w.n_or):
        for p in range(2):
            for mu in range(4):
                schedule.append((oracle.HEATBATH if i == 0 else oracle.OVERRELAX, p, mu))
    # one step = one checkerboard phase, cycling through a sweep's phases in
    # order (8 heat-bath phases, then 8 n_or overrelaxation phases)
    k = 0
    for _ in range(args.warmup):
        L.phase(*schedule[k % len(schedule)], w.seed)
        k += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L.phase(*schedule[k % len(schedule)], w.seed)
        k += 1
    dt = time.perf_counter() - t0
    L.close()
    value = args.steps * Vh / dt
    cores = oracle.get_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (hot start, Philox seed %d)" % w.seed,
            "config": config_of(w),
            "run": {"storage": "FP64 18-real (oracle)", "cores": cores},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one checkerboard phase (%d link updates) per step, cycling "
                                       "through the sweep's HB and OR phases" % Vh},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(w):
    """The workload, identical for both arms (how each arm stores and runs it
    goes in the line's "run" entry)."""
    return {"workload": w.name, "group": "SU(%d)" % w.group, "lattice": "%d^3x%d" % (w.Ns, w.Nt),
            "sites": w.volume, "beta": w.beta, "flux": w.flux,
            "sweep": "1 HB + %d OR + reunitarization + measurement" % w.n_or,
            "l2": "links larger than L2 (no flush between steps)"}


def run_batched(q, stream, world, rank, dist, sweeps, copies=1):
    """Batched scan: 64 uneven SU(2) lattices, `sweeps` sweeps in one
    persistent launch (each rank sweeps its share of the lattices).  With
    copies > 1 the list of lattices is repeated (copy i drawn with seed
    11 + i), so the links outgrow L2 and the sweep streams from HBM."""
    import torch
    from paper_1310_7087_gb300 import dist as qd
    scan = workloads.batch_scan()
    for i in range(1, copies):
        more = workloads.batch_scan(seed=scan.seed + i)
        scan.Ns += more.Ns
        scan.Nt += more.Nt
        scan.beta += more.beta
        scan.flux += more.flux
    mine = qd.shard(scan.volumes, world, rank)
    pick = lambda v: [v[i] for i in mine]
    bt = q.Batch(pick(scan.Ns), pick(scan.Nt), pick(scan.beta), pick(scan.flux),
                 q.QCD_FP32_COMPRESSED, q.QCD_HOT, scan.seed, stream)
    bt.sweep(sweeps, scan.n_or)  # launch shape, graph capture, warm-up
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    bm = bt.sweep(sweeps, scan.n_or)
    g1.record(stream)
    torch.cuda.synchronize()
    bt_ms = qd.max_over_ranks(g0.elapsed_time(g1), "cuda")
    lu_b = qd.sum_over_ranks(float((1 + scan.n_or) * 4 * sum(pick(scan.volumes)) * sweeps), "cuda")
    threads, ctas = q.qcd_batch_get_shape(bt.h)
    waves, wave_bytes = q.qcd_batch_get_waves(bt.h)
    link_bytes = q.qcd_batch_link_bytes(bt.h)
    gbs = lu_b * TRANSFERS_PER_UPDATE * LINK_BYTES[(2, 1)] / (bt_ms / 1e3) / 1e9
    out = {"workload": "batch of %d SU(2) lattices, Ns in {8,12,16,24}, Nt in {4,6,8}, beta in [2.2,2.5], "
                       "flux 0..3 (seeds %d..%d); %d sweeps of 1 HB + %d OR + reunitarization + measurement "
                       "in one launch" % (scan.n, scan.seed, scan.seed + copies - 1, sweeps, scan.n_or),
           "value": lu_b / (bt_ms / 1e3), "unit": UNIT, "ms_total": bt_ms,
           "ms_per_sweep": bt_ms / sweeps, "storage": "FP32 4-real (quaternion)",
           "links_bytes": link_bytes, "effective_gbs": gbs,
           "launch": {"threads_per_cta": threads, "ctas": ctas, "waves": waves, "wave_bytes": wave_bytes},
           "gpu_launches_per_call": 2 + waves,
           "mean_plaquette_last_sweep": float(bm[:, -1, 0].mean())}
    if waves == 1 and link_bytes < 129e6:
        out["note"] = "links fit in L2 (129 MB): effective bandwidth, not HBM"
    else:
        peak, src = load_peaks()
        out["alg_frac_of_hbm"] = gbs / peak
        out["note"] = ("links larger than L2, swept in %d waves of at most %.0f MB (each wave's links stay in L2 "
                       "across the sweeps of its launch): algorithmic bytes (144 B per link update) over the "
                       "sweep time, against the %s HBM peak %.0f GB/s; DRAM carries far less"
                       % (waves, wave_bytes / 1e6, src, peak))
    bt.close()
    return out


def run_paper_lattices(q, stream):
    """Like-for-like context with the paper's Table 1 and its 8^4 comparison:
    SU(2)/SU(3) 8^4 sweeps of 1 HB + reunitarization without measurement, and
    SU(3) 32^4 working sweeps (1 HB + 4 OR + reunitarization + measurement),
    FP32 and FP64.  These lattices fit in L2."""
    import torch
    runs = [("su2_8^4_sweep", 2, 8, 2.3, 0, False, "P: GTX 560 Ti 6e-4 s SP / 1e-3 s DP"),
            ("su3_8^4_sweep", 3, 8, 5.7, 0, False, "P: GTX 560 Ti 1.3e-3 s SP / 4.9e-3 s DP"),
            ("su3_32^4_working_sweep", 3, 32, 6.0, 4, True, "P: GTX 560 Ti 0.56 s SP / 1.17 s DP")]
    out = {}
    for name, group, L, beta, n_or, meas, paper in runs:
        row = {"paper_context": paper}
        for prec, pname in ((q.QCD_FP32_COMPRESSED, "f32"), (q.QCD_FP64_PLAIN, "f64")):
            lat = q.Lattice(group, L, L, beta, 0, prec, q.QCD_HOT, 3, stream)
            lat.sweep(2, n_or, 3)
            torch.cuda.synchronize()
            n = 20
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n):
                q.qcd_sweep(lat.h, 1, n_or, 3)
                if meas:
                    q.qcd_measure(lat.h)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / n
            row[pname] = {"s_per_sweep": ms / 1e3, "lu_per_s": (1 + n_or) * 4 * L ** 4 / (ms / 1e3)}
            lat.close()
        out[name] = row
    return out


def run_on_model(q, stream):
    """O(4) model, 32^4, NHIT = 100: seconds per working sweep (sweep +
    measurement) in FP32 and FP64, as in the paper's Table 1."""
    import torch
    w = workloads.O4_32
    out = {"workload": w.name, "unit": "site hits/s",
           "sweep": "even + odd phase, %d Metropolis hits per site, then measurement" % w.nhit}
    for prec, name in ((q.QCD_FP32_COMPRESSED, "f32"), (q.QCD_FP64_PLAIN, "f64")):
        m = q.ONModel(w.N, w.L, w.L, w.kappa, w.lam, w.delta, prec, q.QCD_HOT, w.seed, stream, w.nhit)
        m.sweep(2, w.seed)
        m.measure()
        torch.cuda.synchronize()
        a0 = m.accepted
        n = 10 if name == "f32" else 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            m.sweep(1, w.seed)
            m.measure()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        out[name] = {"ms_per_working_sweep": ms, "value": w.volume * w.nhit / (ms / 1e3),
                     "acceptance": (m.accepted - a0) / (n * w.volume * w.nhit),
                     "phi2": m.measure()[0]}
        m.close()
    out["paper_context"] = "Table 1, O(4) 32^4: GTX 560 Ti 0.72 s (single) / 0.99 s (double) per working sweep"
    return out


def run_split(q, stream, w):
    """The working-sweep workload on lattices divided along t between device
    memory and host memory (the remedy for lattices larger than the device
    memory): link updates/s with the last 4 and the last 8 of the 16 t-slices
    in host memory, read and written by the GPU over the CPU-GPU link."""
    import torch
    out = {"workload": w.name, "unit": UNIT}
    for nt_dev in (w.Nt * 3 // 4, w.Nt // 2):
        try:
            lat = q.Lattice(w.group, w.Ns, w.Nt, w.beta, w.flux, q.QCD_FP32_COMPRESSED, q.QCD_HOT, w.seed, stream,
                            nt_device=nt_dev)
        except q.QcdError as e:
            out["nt_device_%d" % nt_dev] = {"unavailable": str(e)}
            continue
        dev_b, host_b, got = q.qcd_get_residency(lat.h)
        q.qcd_working_sweep(lat.h, 1, w.n_or, w.seed)
        torch.cuda.synchronize()
        n = 2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            q.qcd_working_sweep(lat.h, 1, w.n_or, w.seed)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        out["nt_device_%d" % got] = {"value": (1 + w.n_or) * 4 * w.volume / (ms / 1e3), "ms_per_step": ms,
                                     "device_link_bytes": dev_b, "host_link_bytes": host_b}
        lat.close()
    return out


def run_flux_scan(q, stream):
    """The SU(3) 32^3 x 8 flux scan (beta 6.0, n in {0, 1, 2, 4}, 500 working
    sweeps of HB + 4 OR each, FP32 links) in both field modes: means and
    binned errors of P, P_s, P_t, Re L, |L|, the bare-link P_s and its
    difference from P_s, plus the working-sweep rate."""
    import torch
    from paper_1310_7087_gb300 import analysis
    w = workloads.SU3_32x8[0]
    fluxes = [v.flux for v in workloads.SU3_32x8]
    out = {"workload": "su3_32^3x8_b6.0, flux n in %s, %d x (1 HB + %d OR + reunitarization + measurement), "
                       "hot start seed %d, FP32 12-real links; first 100 sweeps discarded; [mean, error, tau] "
                       "with errors from the integrated autocorrelation time tau (automatic window)"
                       % (fluxes, w.sweeps, w.n_or, w.seed)}
    for mode, name in ((q.QCD_FIELD_LINKS, "effective_links"), (q.QCD_FIELD_FROZEN, "frozen_boundary")):
        res = analysis.flux_scan(q, fluxes, w.Ns, w.Nt, w.beta, w.sweeps, n_or=w.n_or, seed=w.seed,
                                 n_therm=100, field_mode=mode, stream=stream)
        out[name] = {"n=%d" % n: {k: [round(v[0], 7), round(v[1], 7), round(v[2], 1)] for k, v in st.items()
                                   if isinstance(v, tuple)} for n, st in res.items()}
    # working-sweep rate at n = 1, no host waits inside the timed loop
    lat = q.Lattice(3, w.Ns, w.Nt, w.beta, 1, q.QCD_FP32_COMPRESSED, q.QCD_HOT, w.seed, stream)
    buf = torch.zeros((100, 5), dtype=torch.float64, pin_memory=True)
    q.qcd_working_sweep(lat.h, 3, w.n_or, w.seed)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(100):
        q.qcd_working_sweep(lat.h, 1, w.n_or, w.seed, buf.data_ptr() + 40 * i, wait=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 100
    lat.close()
    out["ms_per_working_sweep"] = ms
    out["value"] = (1 + w.n_or) * 4 * w.volume / (ms / 1e3)
    out["unit"] = UNIT
    # the scan's four chains at once, one lattice and one stream per flux
    # quantum: a 32^3 x 8 phase fills only 1.35 waves of the GPU, so chains
    # queued side by side fill the idle SMs
    streams = [torch.cuda.Stream() for _ in fluxes]
    lats = [q.Lattice(3, w.Ns, w.Nt, w.beta, n, q.QCD_FP32_COMPRESSED, q.QCD_HOT, w.seed, s)
            for n, s in zip(fluxes, streams)]
    n_conc = 50
    cbuf = torch.zeros((len(lats), 1 + n_conc, 5), dtype=torch.float64, pin_memory=True)
    for k, l in enumerate(lats):
        q.qcd_working_sweep(l.h, 3, w.n_or, w.seed, cbuf[k, 0].data_ptr(), wait=False)
    torch.cuda.synchronize()
    e0.record(stream)
    for s in streams:
        s.wait_stream(stream)
    for i in range(n_conc):
        for k, l in enumerate(lats):
            q.qcd_working_sweep(l.h, 1, w.n_or, w.seed, cbuf[k, 1 + i].data_ptr(), wait=False)
    for s in streams:
        stream.wait_stream(s)
    e1.record(stream)
    torch.cuda.synchronize()
    assert bool(torch.all(cbuf[:, :, 0] > 0)), "a queued measurement did not arrive"
    ms_c = e0.elapsed_time(e1)
    for l in lats:
        l.close()
    out["concurrent_chains"] = {"chains": len(lats), "sweeps_each": n_conc, "ms_total": ms_c,
                                "value": len(lats) * n_conc * (1 + w.n_or) * 4 * w.volume / (ms_c / 1e3),
                                "unit": UNIT}
    out["note"] = ("links (50 MB) fit in L2; effective-link observables must not depend on n (change of "
                   "variables), the bare P_s and the frozen-boundary runs show the field")
    return out


def run_su2_large(q, stream):
    """SU(2) on the benchmark's 64^3 x 16 lattice (links 268 MB FP32, beyond
    L2), working sweeps of 1 HB + 1 OR + reunitarization + measurement: the
    SU(2) FP32 and FP64 phase kernels against the HBM roofline (144 / 288 B of
    algorithmic traffic per link update)."""
    import torch
    Ns, Nt, beta = 64, 16, 2.4
    V = Ns ** 3 * Nt
    peak, src = load_peaks()
    out = {"workload": "su2_64^3x16_b2.4_n1, working sweeps of 1 HB + 1 OR + reunitarization + measurement",
           "unit": UNIT}
    for prec, name in ((q.QCD_FP32_COMPRESSED, "f32"), (q.QCD_FP64_PLAIN, "f64")):
        lat = q.Lattice(2, Ns, Nt, beta, 1, prec, q.QCD_HOT, 3, stream)
        q.qcd_working_sweep(lat.h, 2, 1, 3)
        q.qcd_set_profiling(lat.h, True)
        torch.cuda.synchronize()
        n = 20
        buf = torch.zeros((n, 5), dtype=torch.float64, pin_memory=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(n):
            q.qcd_working_sweep(lat.h, 1, 1, 3, buf.data_ptr() + 40 * i, wait=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        pm, pn = q.qcd_get_profile(lat.h)
        q.qcd_set_profiling(lat.h, False)
        lat.close()
        hb_ms = pm[0] / max(1, pn[0])
        alg = TRANSFERS_PER_UPDATE * LINK_BYTES[(2, prec)] * (V // 2)
        out[name] = {"value": 2 * 4 * V / (ms / 1e3), "ms_per_working_sweep": ms,
                     "heatbath_ms_per_launch": hb_ms,
                     "heatbath_alg_gbs": alg / (hb_ms / 1e3) / 1e9,
                     "heatbath_frac_of_hbm": alg / (hb_ms / 1e3) / 1e9 / peak,
                     "kernel_ms": [round(m / n, 4) for m in pm], "kernel_launches": [int(c) for c in pn]}
    out["peak_source"] = src
    return out


def run_su2_single_lattices(q, stream, batched_value):
    """Same group and the same work as the batched scan, swept one lattice
    at a time: the 64 SU(2) lattices of the scan as single lattices, FP64 and
    FP32 storage, each working sweep (1 HB + 1 OR + reunitarization +
    measurement) enqueued without host waits."""
    import torch
    scan = workloads.batch_scan()
    out = {"workload": "the %d SU(2) lattices of the batched scan, one working sweep of each per step, "
                       "one lattice at a time" % scan.n}
    lu = (1 + scan.n_or) * 4 * sum(scan.volumes)
    for prec, name in ((q.QCD_FP64_PLAIN, "f64_plain"), (q.QCD_FP32_COMPRESSED, "f32_single")):
        lats = [q.Lattice(2, ns, nt, b, n, prec, q.QCD_HOT, scan.seed, stream)
                for ns, nt, b, n in zip(scan.Ns, scan.Nt, scan.beta, scan.flux)]
        buf = torch.zeros((len(lats), 5), dtype=torch.float64, pin_memory=True)
        for k, lat in enumerate(lats):
            q.qcd_working_sweep(lat.h, 1, scan.n_or, scan.seed)
        torch.cuda.synchronize()
        steps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            for k, lat in enumerate(lats):
                q.qcd_working_sweep(lat.h, 1, scan.n_or, scan.seed, buf.data_ptr() + 40 * k, wait=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        for lat in lats:
            lat.close()
        out[name] = {"value": lu / (ms / 1e3), "unit": UNIT, "ms_per_scan_sweep": ms}
    out["batched_f32_over_single_f64"] = batched_value / out["f64_plain"]["value"]
    out["batched_f32_over_single_f32"] = batched_value / out["f32_single"]["value"]
    return out


def main():
    args = parse()
    w = workloads.SU3_64x16
    if args.Ns or args.Nt:
        import dataclasses
        Ns, Nt = args.Ns or w.Ns, args.Nt or w.Nt
        w = dataclasses.replace(w, Ns=Ns, Nt=Nt, name="su3_%d^3x%d_b%g_n%d" % (Ns, Nt, w.beta, w.flux))
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1310_7087_gb300 import build
    build.build()
    import paper_1310_7087_gb300 as q

    stream = torch.cuda.current_stream()
    if args.batch_only:
        out = run_batched(q, stream, world, rank, dist, args.steps, args.batch_copies)
        if rank == 0:
            print(json.dumps(dict(out, metric=METRIC, n_gpus=world, steps=args.steps, warmup=1,
                                  higher_is_better=True, scaling="weak", dtype="f32", data="synthetic")),
                  flush=True)
        return 0
    seed = w.seed + 1000 * rank
    prec = q.QCD_FP64_PLAIN if args.storage == "fp64" else q.QCD_FP32_COMPRESSED
    lat = q.Lattice(w.group, w.Ns, w.Nt, w.beta, w.flux, prec, q.QCD_HOT, seed, stream)
    h = lat.h
    lu_per_step = (1 + w.n_or) * 4 * w.volume

    # One step = one working sweep: sweep + measurement (fused into the last
    # OR pass), its five measured doubles read back into pinned host memory.
    # Steps are queued without a host wait between them, as a Monte Carlo run
    # queues its sweeps; the results are checked once the timed steps are done.
    meas = torch.zeros((args.warmup + 2 + args.steps, 5), dtype=torch.float64, pin_memory=True)
    row = [0]

    def step():
        q.qcd_working_sweep(h, 1, w.n_or, seed, meas.data_ptr() + row[0] * meas.stride(0) * 8, wait=False)
        row[0] += 1

    for _ in range(args.warmup):
        step()
    # the two alternating instances of the profiled sweep graph are captured
    # before the timed region; enabling again restarts the totals
    q.qcd_set_profiling(h, True)
    step()
    step()
    q.qcd_set_profiling(h, True)
    clocks = ClockSampler(local)
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    assert bool(torch.all(meas[:row[0], 0] > 0)), "a queued measurement did not arrive"
    last = (meas[row[0] - 1, :3].tolist(), meas[row[0] - 1, 3:].tolist())
    clocks.stop()
    if dist:
        dist.barrier()
    t_ms = e0.elapsed_time(e1)
    prof_ms, prof_n = q.qcd_get_profile(h)
    q.qcd_set_profiling(h, False)
    if dist:
        t = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    value = lu_per_step * args.steps * world / (t_ms / 1e3)

    # roofline of the dominant kernel (largest share of the timed kernel time)
    names = ["heatbath_phase", "overrelax_phase", "last_pass_with_reunit", "measure"]
    dom = max(range(2), key=lambda k: prof_ms[k])
    per_launch_ms = prof_ms[dom] / max(1, prof_n[dom])
    link_b = LINK_BYTES[(w.group, prec)]
    alg_bytes = TRANSFERS_PER_UPDATE * link_b * (w.volume // 2)
    peak, peak_src = load_peaks()
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": ncu_traffic(names[dom], w.name), "kernel": names[dom],
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src if peak_src == "measured"
                else "fallback 6.8 TB/s",
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": per_launch_ms,
                "kernel_ms": {n: round(m, 3) for n, m in zip(names, prof_ms)},
                "kernel_launches": {n: int(c) for n, c in zip(names, prof_n)}}
    # link updates per second of the heat-bath and overrelaxation kernels alone
    # (V/2 updates per phase launch), whole job
    rates = {k: world * (w.volume // 2) / (prof_ms[i] / max(1, prof_n[i]) / 1e3) if prof_n[i] else None
             for k, i in (("hb", 0), ("or", 1))}

    # end to end through the C ABI: every step uploads its configuration from
    # pinned host memory, sweeps it and reads its measurement back to pinned
    # host memory.  Two lattices on two streams alternate, so one step's
    # upload overlaps the other's sweep (a two-deep pipeline); an event chain
    # keeps the sweeps themselves in order, one at a time (two sweeps running
    # side by side split L2 between two lattices and ran 3 % slower).
    nbytes = q.qcd_link_bytes(h)
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    q.qcd_copy_links_out(h, host.data_ptr(), nbytes)
    # as many timed steps as the device-timed pass (at least 40): the first
    # step's upload has no sweep before it to hide behind
    e2e_steps, e2e_warmup = max(40, args.steps), 4
    stream2 = torch.cuda.Stream()
    lat2 = q.Lattice(w.group, w.Ns, w.Nt, w.beta, w.flux, prec, q.QCD_HOT, seed, stream2)
    pipe = [h, lat2.h]
    results = torch.zeros((e2e_warmup + e2e_steps, 5), dtype=torch.float64, pin_memory=True)
    for hh in pipe:  # graphs and launch shape in place before timing
        q.qcd_copy_links_in(hh, host.data_ptr(), nbytes)
        q.qcd_working_sweep(hh, 1, w.n_or, seed)
    torch.cuda.synchronize()
    streams = [stream, stream2]
    done = [torch.cuda.Event(), torch.cuda.Event()]

    # device events around every timed sweep: where the end-to-end time goes
    sweep_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(e2e_steps)]

    def pipeline(first, n, events=None):
        for i in range(first, first + n):
            k = i % 2
            q.qcd_copy_links_in(pipe[k], host.data_ptr(), nbytes)
            if i > first:
                streams[k].wait_event(done[1 - k])
            if events:
                events[i - first][0].record(streams[k])
            q.qcd_working_sweep(pipe[k], 1, w.n_or, seed, results.data_ptr() + i * results.stride(0) * 8,
                                wait=False)
            done[k].record(streams[k])
            if events:
                events[i - first][1].record(streams[k])

    # untimed warm-up steps of the same pipeline on the same buffers (the first
    # pipelined steps of a fresh process measured up to 20 % slower)
    pipeline(0, e2e_warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks_e2e = ClockSampler(local)
    time.sleep(0.3)
    clocks_e2e.start()
    t0 = time.perf_counter()
    pipeline(e2e_warmup, e2e_steps, sweep_ev)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    clocks_e2e.stop()
    assert bool(torch.all(results[:, 0] > 0)), "a pipelined measurement did not arrive"
    sweep_ms = [a.elapsed_time(b) for a, b in sweep_ev]
    first_to_last_ms = sweep_ev[0][0].elapsed_time(sweep_ev[-1][1])
    lat2.close()
    if dist:
        t = torch.tensor([t_e2e], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t.item())
    e2e = {"value": lu_per_step * e2e_steps * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": 5 * 8, "steps": e2e_steps,
           "sweep_ms_mean": sum(sweep_ms) / len(sweep_ms), "sweep_ms_max": max(sweep_ms),
           "first_to_last_sweep_ms": first_to_last_ms, "host_ms": 1e3 * t_e2e,
           "clocks": clocks_e2e.summary(),
           "pipeline": "each step uploads a configuration in the library's device storage layout "
                       "(qcd_copy_links_in of the qcd_link_bytes bytes qcd_copy_links_out gave) from pinned "
                       "host memory and reads its five measured doubles back (qcd_working_sweep into pinned "
                       "memory); two lattices on two streams: upload of one step overlaps the sweep of the "
                       "other; sweeps ordered one after another by events; 4 untimed warm-up steps of the same "
                       "pipeline before the timed ones"}

    extras = {}
    if not args.no_extras:
        # FP64-plain single lattice, same workload, for the FP32-vs-FP64 comparison
        lat64 = q.Lattice(w.group, w.Ns, w.Nt, w.beta, w.flux, q.QCD_FP64_PLAIN, q.QCD_HOT, seed, stream)
        q.qcd_sweep(lat64.h, 1, w.n_or, seed)
        q.qcd_measure(lat64.h)
        q.qcd_set_profiling(lat64.h, True)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n64 = 2
        f0.record(stream)
        for _ in range(n64):
            q.qcd_sweep(lat64.h, 1, w.n_or, seed)
            q.qcd_measure(lat64.h)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / n64
        pm, pn = q.qcd_get_profile(lat64.h)
        extras["fp64_plain"] = {"value": lu_per_step / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                                "storage": "FP64 18-real", "bound": "fp64 alu",
                                "kernel_ms_per_step": {n: round(m / n64, 3) for n, m in zip(names, pm)},
                                "fp32_speedup": (lu_per_step * args.steps / (t_ms / 1e3)) /
                                                (lu_per_step / (ms64 / 1e3))}
        if pn[1]:
            or_ms = pm[1] / pn[1]
            tf = FP64_OR_FLOPS * (w.volume // 2) / (or_ms / 1e3) / 1e12
            try:
                peak64, src64 = q.qcd_probe_fp64_rate(stream) / 1e12, "measured in this run (qcd_probe_fp64_rate)"
            except q.QcdError as e:
                peak64, src64 = FP64_PEAK_TFLOPS_NOMINAL, "nominal GB300 FP64 (probe failed: %s)" % e
            extras["fp64_plain"]["roofline"] = {
                "bound": "alu", "kernel": "overrelax_phase", "unit": "TFLOP/s", "achieved": tf,
                "peak": peak64, "frac": tf / peak64, "flops_per_update": FP64_OR_FLOPS,
                "avg_launch_ms": or_ms, "peak_source": src64,
                "nominal_peak": FP64_PEAK_TFLOPS_NOMINAL}
        lat64.close()

        extras["batched"] = run_batched(q, stream, world, rank, dist, workloads.batch_scan().sweeps)
        extras["batched_beyond_l2"] = run_batched(q, stream, world, rank, dist, 20, copies=8)
        extras["su2_same_work_single_lattices"] = run_su2_single_lattices(q, stream, extras["batched"]["value"])
        extras["su2_64x16"] = run_su2_large(q, stream)
        extras["c3_flux_scan"] = run_flux_scan(q, stream)
        extras["o4_model"] = run_on_model(q, stream)
        extras["paper_lattices"] = run_paper_lattices(q, stream)
        extras["split_residency"] = run_split(q, stream, w)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_oracle(w)

    launches = int(sum(prof_n))
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.storage == "fp64" else "f32",
                "data": "synthetic: hot start (Haar links from Philox seed %d), no dataset" % w.seed,
                "config": config_of(w),
                "run": {"storage": "FP64 18-real" if args.storage == "fp64"
                        else "FP32 12-real (rows 1-2, row 3 rebuilt)",
                        "parallelism": "replicas" if world > 1 else "single GPU", "block": q.qcd_get_block(h)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks.summary(),
                "hb_lu_per_s": rates["hb"], "or_lu_per_s": rates["or"],
                "sweeps_per_s": 1e3 * args.steps / t_ms * world,
                "gpu_launches": launches, "last_measurement": {"plaquette": last[0], "polyakov": last[1]},
                **extras}
        print(json.dumps(line), flush=True)
    lat.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
