"""Benchmark: exact Breit-Wheeler collision detection, 2 x 1,048,576 photons.

One benchmark step = one full run of the head-on workload: 64 time steps of
5 fs, each a hierarchy build of both beams plus the collision step (dual
traversal, FP32 narrow phase, FP64 band re-test, yield), inputs resident in
HBM.  The metric is the narrow-phase photon-pair tests per second: photon
pairs that reach the exact closest-approach test (the work the method
does after the hierarchy has pruned).  Collided pairs/s and the all-pairs
equivalent N_A * N_B * time steps per second are reported beside it as
context.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the path has no exchange step); the value is the units of all ranks over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1608_01125_gb300 import synth  # noqa: E402

METRIC = "narrow-phase photon-pair tests/s at 2x1M (photon pairs given the exact test per second)"
UNIT = "pair-tests/s"
# the oracle's CPU samples: every 4th time step (a systematic sample of the
# run's busy and empty steps), all host cores; single-threaded (as the paper
# ran) on one busy and one empty step
CPU_STEP_STRIDE = 4
SINGLE_THREAD_STEPS = (4, 36)
FALLBACK_HBM_GBS = 6800.0
PHASES = ("propagate", "sort", "gather", "emit", "refit", "expand", "traverse", "narrow", "band",
          "yield")
# FP32 operations of the narrow test's prefix (threshold and quick miss), which
# decides most photon pairs: the invariant s and its bound (13), the relative
# position and direction and their products (15), the reciprocal and the
# closest approach (8), the position sum and the quick-miss comparisons (11)
NARROW_OPS_PER_TEST = 47
# GB300 FP32 lanes: 152 SMs x 128 per SM at the 2070 MHz maximum SM clock
FP32_OPS_PEAK = 152 * 128 * 2.07e9


def algorithmic_bytes(phase: str, na: int, nb: int, key_bits: tuple, hits: float, band: float):
    """Bytes one launch of a phase must move at least (per beam launches use
    that beam's size; traversal and later phases cover both beams)."""
    n = na + nb
    if phase == "propagate":   # p0, d (6 doubles) and the FP32 direction in; x, y, z + key + index out
        return 48 + 16 + 12 + 12, "photon"
    if phase == "sort":        # per pass: key + index read and written
        return 24, "photon-pass"
    if phase == "gather":      # index, random float4 x2 read, float4 x2 written
        return 4 + 32 + 32, "photon"
    if phase == "emit":        # keys read, child refs + counts + parent written
        return 8 + 16 + 4, "photon"
    if phase == "refit":       # sorted SoA, parent links and ranges read; two child boxes per node
        return 32 + 8 + 4 + 4 + 48, "photon"
    if phase == "traverse":    # node records of both trees once + the leaf pairs written
        return 64, "photon"
    if phase == "narrow":      # sorted photon records once + the leaf pairs read + output pairs
        return 32, "photon"
    return 8, "pair"


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def src_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1608_01125_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(kernel: str):
    """The fields of the committed ncu summary's line for `kernel` (DRAM bytes
    per launch, and what the capture was: time steps, knobs, the algorithmic
    bytes of the same launches), if the kernel sources have not changed since it
    was taken; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    cur = src_hash()
    for line in open(p):
        if line.startswith("#"):
            continue
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("phase") == kernel and f.get("src") == cur and "bytes_per_launch" in f:
            return f
    return None


class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(float(r[2]) for r in rows),
                "power_w_median": statistics.median(float(r[3]) for r in rows if _isnum(r[3])),
                "samples": len(rows), "reasons": reasons}


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


# ------------------------------------------------------------------ oracle leg


def oracle_sample(wl, a, b, steps, threads):
    """The FP64 k-d-tree oracle over the given time steps: (seconds, hits,
    narrow-phase tests)."""
    import oracle
    t0 = time.perf_counter()
    hits = tests = 0
    for k in steps:
        _, r = oracle.tree(a, b, k, wl.dt, wl.kappa, nthreads=threads, cap=1 << 22)
        hits += r["count"]
        tests += r["tests"]
    return time.perf_counter() - t0, hits, tests


def cpu_baseline(wl, a, b, first=0, nsteps=None):
    threads = os.cpu_count() or 1
    nsteps = nsteps or wl.steps
    steps = list(range(first, first + nsteps, CPU_STEP_STRIDE))
    dt, hits, tests = oracle_sample(wl, a, b, steps, threads)
    st_steps = [k for k in SINGLE_THREAD_STEPS if first <= k < first + nsteps] or steps[:1]
    dt1, _, tests1 = oracle_sample(wl, a, b, st_steps, 1)
    return {"value": tests / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"FP64 k-d-tree oracle (leaf size 8), every {CPU_STEP_STRIDE}th time step "
                      f"({len(steps)} of the {nsteps}-step run: {steps[0]}, {steps[1] if len(steps) > 1 else ''}"
                      f"...), {threads} threads, {dt:.1f} s, {tests} narrow-phase tests, {hits} hits",
            "all_pairs_per_s": wl.a.n * wl.b.n * len(steps) / dt,
            "single_thread": {"value": tests1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"time steps {st_steps}, one thread, {dt1:.1f} s, "
                                        f"{tests1} narrow-phase tests"}}


# FP64 operations per hit of the pair products, counted from the kernel: 26
# for the photons' sums, the invariant mass and the CoM momentum, ~16 for the
# direction (1.27 Marsaglia tries of 2 draws), 4 divisions, 2 x 16 for the two
# boosts; 3 square roots; divisions and square roots counted as one each
PAIR_FP64_OPS = 26 + 16 + 4 + 32 + 3
FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64, nominal (no measured figure here)


def pair_products_timing(col, A, B, stream, step=2, seed=2024, reps=5):
    """The pair products (electron and positron of each collision) of the
    collision-peak step's hits: device time per call with CUDA events."""
    import torch

    from paper_1608_01125_gb300 import binding
    h, _ = col.step_hits(step)
    hits = torch.as_tensor(h.astype("uint32").view("int32"), device=A["px"].device).reshape(-1, 2)
    out = binding.pair_products(A, B, hits, seed)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        binding.pair_products(A, B, hits, seed, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = min(ts)
    n = int(hits.shape[0])
    flops = n * PAIR_FP64_OPS / (ms / 1e3) / 1e12
    return {"step": step, "hits": n, "ms": ms, "hits_per_s": n / (ms / 1e3),
            "roofline": {"bound": "alu", "achieved": flops, "peak": FP64_NOMINAL_TFLOPS,
                         "unit": "FP64 TFLOP/s", "peak_source": "nominal",
                         "frac": flops / FP64_NOMINAL_TFLOPS,
                         "bytes_per_hit": 8 + 2 * 32 + 64}}


# Algorithmic bytes per hit of a depletion call: the t* gather (hit 8, two photons'
# p0 and direction 96, their remaining weights 16, key/state/delta written 17), one
# round over every hit (state 1 + hit 8 + key 8 read three times, rem 16, four slot
# reads 24 and resets 24, delta 8) and the sum (8).  Later rounds touch the open hits
# only and are not counted.
DEP_BYTES_PER_HIT = (8 + 96 + 16 + 17) + (3 * 17 + 16 + 24 + 24 + 8) + 8


def depletion_timing(col, stream, steps, peak, peak_src, host=None):
    """Depletion in time order over a whole run (unit weights, what is left
    carried from step to step).  The run's hit lists are made first (every step
    built and collided, not timed) and stay on the device.  Then the depletion
    of every step with hits is enqueued back to back (trilens_deplete_step_async,
    one record per step, read after the run) between two CUDA events on the
    launching stream: the device time of the run's depletion.  Beside it the
    synchronous call (trilens_deplete_step) step by step, each between two
    events: it waits for its result, so that sum holds a host round trip per
    step.  Each is done three times; the last is reported.  With host = (beam a,
    beam b, dt, kappa) as numpy, the oracle then depletes the same hit lists on
    the host cores (timed, and its pairs compared with the GPU's)."""
    import torch

    from paper_1608_01125_gb300 import binding
    dev = col.a["px"].device
    na, nb = col.a["px"].numel(), col.b["px"].numel()
    cap = 1 << 21
    buf = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    lists = []
    for k in steps:
        col.build(k)
        while True:
            try:
                n = col.collide(k, buf)
                break
            except binding.TrilensError as e:
                if e.code != binding.ERR_CAPACITY:
                    raise
                cap = e.needed + 1024
                buf = torch.empty((cap, 2), dtype=torch.int32, device=dev)
        if n:
            lists.append((k, buf[:n].clone(), n))
    hits = sum(n for _, _, n in lists)
    delta = torch.empty(max([n for _, _, n in lists] + [1]), dtype=torch.float64, device=dev)
    out = torch.zeros((max(len(lists), 1), 4), dtype=torch.int64, device=dev)
    for rep in range(3):
        ra = torch.ones(na, dtype=torch.float64, device=dev)
        rb = torch.ones(nb, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for q, (k, h, n) in enumerate(lists):
            col.deplete_step_async(k, h, n, ra, rb, delta, out[q])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    recs = binding.deplete_record(out)[: len(lists)]
    assert all(r["status"] == 0 for r in recs), recs
    used = int((ra == 0).sum().item())
    acc = sum(r["accepted"] for r in recs)
    made = sum(r["transferred"] for r in recs)
    rounds = [r["rounds"] for r in recs]
    for rep in range(3):
        ra = torch.ones(na, dtype=torch.float64, device=dev)
        rb = torch.ones(nb, dtype=torch.float64, device=dev)
        sync_ms = wall = 0.0
        sync_acc = 0
        for k, h, n in lists:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            r = col.deplete_step(k, h, n, ra, rb, delta)
            e1.record(stream)
            torch.cuda.synchronize()
            wall += 1e3 * (time.perf_counter() - t0)
            sync_ms += e0.elapsed_time(e1)
            sync_acc += r["accepted"]
    assert sync_acc == acc
    cpu = None
    if host is not None:
        import oracle
        a_np, b_np, dt, kappa = host
        o_ra, o_rb = np.ones(na), np.ones(nb)
        o_made = 0
        host_lists = [(k, h.cpu().numpy().view(np.uint32)) for k, h, _ in lists]
        t0 = time.perf_counter()
        for k, h in host_lists:
            t = oracle.hit_times(a_np, b_np, k, dt, kappa, h)
            d, o_ra, o_rb = oracle.deplete(k, t, h, o_ra, o_rb)
            o_made += int((d > 0).sum())
        cpu_s = time.perf_counter() - t0
        cpu = {"kind": "oracle", "cores": 1, "ms_per_run": 1e3 * cpu_s,
               "hits_per_s": hits / cpu_s, "pairs_made": o_made, "equal_to_gpu": o_made == acc,
               "sample": "the same run's hit lists, every step (t* of every hit, then the "
                         "time-ordered sweep)"}
    achieved = DEP_BYTES_PER_HIT * hits / (ms / 1e3) / 1e9
    return {"time_steps": len(steps), "hits": hits, "pairs_made": acc, "transferred": made,
            "photons_used_up_a": used, "ms_per_run": ms, "hits_per_s": hits / (ms / 1e3),
            "sync_ms_per_run": sync_ms, "sync_wall_ms_per_run": wall,
            "rounds_max": max(rounds or [0]),
            "rounds_per_step_with_hits": statistics.mean(rounds or [0]),
            "steps_with_hits": len(lists),
            # one cooperative launch (and a 16-byte memset) per step with hits
            "launches_per_run": len(lists),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                         "bytes_per_hit": DEP_BYTES_PER_HIT},
            "cpu_baseline": cpu}


def ip_regime_timing(dev, stream, reps=3, cpu=True):
    """IP regime on the 2 x 16384-MP head-on workload (mean weight 100): the marking
    of the MPs that can collide (all MP pairs: FP32 pre-test, FP64 decision), counting
    and writing the real photons, and the exact run over the real photons (one
    captured graph).  Device times with CUDA events; the best of `reps` repetitions
    after one warm-up.  With cpu, the oracle decides every real-photon pair of 64 MP
    pairs sampled from the marked ones at the collision-peak step (timed on one host
    core)."""
    import torch

    from paper_1608_01125_gb300 import binding
    wl = synth.ip_headon()
    a_np, b_np = synth.beams(wl)
    h = synth.IP_CUBE_UM
    A, B = binding.to_device(a_np, dev), binding.to_device(b_np, dev)

    def timed(fn):
        best, out = None, None
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None or ms < best else best
        return best, out

    mark_ms, marks = timed(lambda: binding.swarm_mark(A, B, h, h, wl.dt, wl.kappa, 0, wl.steps,
                                                      stream))
    split_ms, sp = timed(lambda: binding.swarm_split(A, B, h, h, wl.dt, wl.kappa, 0, wl.steps,
                                                     stream))
    na, nb = int(sp["a"]["px"].numel()), int(sp["b"]["px"].numel())
    col = binding.Collider(sp["a"], sp["b"], wl.dt, wl.kappa, precision=binding.FP32_BAND,
                           stream=stream)
    run_ms, r = timed(lambda: col.run(0, wl.steps))
    col.close()
    pairs = wl.a.n * wl.b.n
    cpu_line = None
    if cpu:
        import oracle
        ma = np.nonzero(marks[0].cpu().numpy())[0]
        mb = np.nonzero(marks[1].cpu().numpy())[0]
        rng = np.random.default_rng(7)
        ia, jb = rng.choice(ma, 64), rng.choice(mb, 64)
        sub = lambda beam, i: {k: v[i:i + 1].copy() for k, v in beam.items()}  # noqa: E731
        tests = 0
        t0 = time.perf_counter()
        for i, j in zip(ia, jb):
            oracle.ip_bruteforce(sub(a_np, i), sub(b_np, j), h, h, 2, wl.dt, wl.kappa)
            tests += int(a_np["w"][i]) * int(b_np["w"][j])
        cpu_s = time.perf_counter() - t0
        cpu_line = {"kind": "oracle", "cores": 1, "real_pair_tests_per_s": tests / cpu_s,
                    "sample": f"64 marked MP pairs at step 2, {tests} real-photon pairs"}
    return {"workload": wl.name, "macro_photons_per_beam": wl.a.n, "cube_um": h,
            "time_steps": wl.steps, "real_photons": [na, nb],
            "marked": [int(marks[0].sum().item()), int(marks[1].sum().item())],
            "mark_ms": mark_ms, "split_ms": split_ms, "run_ms": run_ms,
            "total_ms": split_ms + run_ms, "hits_per_run": r["count"],
            "real_pair_tests_per_s": na * nb * wl.steps / ((split_ms + run_ms) / 1e3),
            # all MP pairs are covered; most are skipped (both MPs already marked) or
            # rejected by the FP32 pre-test, so no single arithmetic roofline applies
            "mark_mp_pairs_per_s": pairs / (mark_ms / 1e3),
            "cpu_baseline": cpu_line}


def crossing_timing(dev, stream, peak, peak_src, steps=(120, 129, 141, 160)):
    """The large exact workload (2 x 5e7 photons crossing at 90 degrees, Gamma
    energies, 2 fs steps): a few of its busy time steps built and collided one
    at a time with per-phase device times (CUDA events).  Here the two
    hierarchies (2 x 5e7 x 64 B of node records) are far larger than the L2,
    so the traversal's HBM fraction is measured where it can matter.  The
    hit counts of steps 129, 141 and 160 are the oracle's (the GPU tests
    compare their checksums)."""
    import torch

    from paper_1608_01125_gb300 import binding
    wl = synth.crossing90_5e7()
    a_np, b_np = synth.beams(wl)
    A, B = binding.to_device(a_np, dev), binding.to_device(b_np, dev)
    del a_np, b_np
    col = binding.Collider(A, B, wl.dt, wl.kappa, precision=binding.FP32_BAND, stream=stream)
    tuned = col.autotune([steps[1]], os.path.join(ROOT, "paper_1608_01125_gb300",
                                                  "_tuning_cache.json"))
    col.timing(True)
    rows = []
    for k in steps:
        col.build(k)
        col.phase_ms(reset=True)
        col.collide(k)
        torch.cuda.synchronize()
        col.phase_ms(reset=True)
        col.build(k)  # timed: the build and the collision of step k
        col.collide(k)
        ph, _ = col.phase_ms(reset=True)
        st = col.stats()
        rows.append({"step": k, **{p: round(ph[p], 4) for p in PHASES}, "hits": st["count"],
                     "narrow_tests": st["narrow_tests"], "node_tests": st["node_tests"],
                     "leaf_pairs": st["leaf_pairs"]})
    col.timing(False)
    col.close()
    n_ab = wl.a.n + wl.b.n
    tt = sum(r["traverse"] for r in rows)
    tbytes = sum(64.0 * n_ab + 8.0 * r["leaf_pairs"] for r in rows)
    ach = tbytes / (tt / 1e3) / 1e9
    tot = sum(sum(r[p] for p in PHASES) for r in rows)
    return {"workload": wl.name, "photons_per_beam": wl.a.n, "time_steps_timed": list(steps),
            "tuning": tuned, "ms_per_step": tot / len(rows), "per_step": rows,
            "narrow_tests_per_s": sum(r["narrow_tests"] for r in rows) / (tot / 1e3),
            "collided_pairs_per_s": sum(r["hits"] for r in rows) / (tot / 1e3),
            "traverse_roofline": {"bound": "hbm", "achieved": ach, "peak": peak,
                                  "peak_source": peak_src, "unit": "GB/s", "frac": ach / peak,
                                  "algorithmic_bytes": tbytes, "ms": tt,
                                  "unit_of_work": "node records of both trees once, leaf pairs "
                                                  "written, per step"}}


def run_reference(args, wl):
    """The oracle as the reference arm: bench step q times the time steps
    {j, j + 16, j + 32, j + 48} of the run with j = q mod 16, so that 16 bench
    steps cover every time step once and any K steps keep the run's mix of
    busy and empty steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    a, b = synth.beams(wl)
    threads = os.cpu_count() or 1
    first, nsteps = args.first_step, (args.time_steps or wl.steps)
    stride = max(nsteps // 4, 1)
    sample = lambda q: [first + (q % stride) + m * stride  # noqa: E731
                        for m in range(4) if (q % stride) + m * stride < nsteps]
    for q in range(args.warmup):
        oracle_sample(wl, a, b, sample(q)[-1:], threads)
    total = 0.0
    tests = hits = 0
    for q in range(args.steps):
        dt, h, t = oracle_sample(wl, a, b, sample(q), threads)
        total += dt
        tests += t
        hits += h
    value = tests / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": config_of(wl, L2_NOTE, nsteps, first),
            "collided_pairs_per_s": hits / total,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"bench step q = time steps q mod {stride} + {{0, {stride}, "
                                       f"{2 * stride}, {3 * stride}}} of the {nsteps}-step run "
                                       f"(FP64 k-d-tree oracle, leaf size 8, {threads} threads)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def slowest_rank_ms(ms: float, world: int, device=None) -> float:
    """The largest of every rank's time (ranks run replicas; the job ends with
    the slowest).  A collective only when there are several ranks."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units all ranks processed per second of the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


L2_NOTE = "GPU: L2 flushed (256 MiB write) before every timed step"


def config_of(wl, l2, nsteps=None, first=0):
    return {"workload": wl.name, "photons_per_beam": wl.a.n, "time_steps": nsteps or wl.steps,
            "first_step": first, "dt_fs": wl.dt, "kappa": wl.kappa,
            "precision": "fp32 + fp64 band", "l2": l2, "parallelism": "replicas"}


# ------------------------------------------------------------------ GPU leg


def run_ours(args, wl):
    import torch
    import torch.distributed as dist

    from paper_1608_01125_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    a_np, b_np = synth.beams(wl, seed=wl.seed + rank)
    A = binding.to_device(a_np, dev)
    B = binding.to_device(b_np, dev)
    col = binding.Collider(A, B, wl.dt, wl.kappa, precision=binding.FP32_BAND, stream=stream)

    first, nsteps = args.first_step, (args.time_steps or wl.steps)
    time_steps = range(first, first + nsteps)

    def stepwise_run():
        # build + collide one step at a time (a host check after every step)
        hits = tests = band = 0
        for k in time_steps:
            col.build(k)
            hits += col.collide(k)
            st = col.stats()
            tests += st["narrow_tests"]
            band += st["band"]
        return hits, tests, band

    work = {}

    def graph_run():
        # the same steps as one captured CUDA graph (trilens_run)
        r = col.run(first, nsteps)
        work.update(node_tests=r["node_tests"], leaf_pairs=r["leaf_pairs"])
        return r["count"], r["narrow_tests"], r["band"]

    if args.knobs:  # fixed knobs (profiling): bucket, stack depth, warps per block, budget
        col.set_tuning(*[int(x) for x in args.knobs.split(",")])
        tuned = col.tuning()
    elif args.tune:
        tuned = col.autotune([2, 4, 40], os.path.join(ROOT, "paper_1608_01125_gb300",
                                                      "_tuning_cache.json"))
    else:
        tuned = col.tuning()
    for _ in range(max(args.warmup, 0)):
        graph_run()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = []
    hits = tests = band = 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.zero_()  # L2 flush, outside the timed events
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h, t, bd = graph_run()
            e1.record(stream)
            evs.append((e0, e1))
            hits += h
            tests += t
            band += bd
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    # per-phase device times: the same runs step by step, with CUDA events
    # around every phase on the launching stream
    col.timing(True)
    col.phase_ms(reset=True)
    sw_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stepwise_run()
        e1.record(stream)
        torch.cuda.synchronize()
        sw_ms.append(e0.elapsed_time(e1))
    phase_ms, launches = col.phase_ms(reset=True)
    # the traversal step by step: its device time per time step, to give the
    # roofline of the busy steps (where the bunches cross) beside the run's average
    per_step = []
    for k in time_steps:
        col.build(k)
        col.phase_ms(reset=True)
        col.collide(k)
        ph, _ = col.phase_ms(reset=True)
        st = col.stats()
        per_step.append(dict(step=k, traverse=ph["traverse"], narrow=ph["narrow"],
                             tests=st["narrow_tests"], hits=st["count"], band=st["band"],
                             leaves=st["leaf_pairs"]))
    col.timing(False)
    pairs = pair_products_timing(col, A, B, stream) if rank == 0 else None
    depl = (depletion_timing(col, stream, list(time_steps), *read_peaks(),
                             host=None if args.no_cpu_baseline else (a_np, b_np, wl.dt, wl.kappa))
            if rank == 0 and not args.no_depletion else None)
    ipr = (ip_regime_timing(dev, stream, cpu=not args.no_cpu_baseline)
           if rank == 0 and not args.no_ip else None)
    crossing = (crossing_timing(dev, stream, *read_peaks())
                if rank == 0 and not args.no_crossing else None)
    # the learned statistical regime on a 2 x 1e6 sample of the statistical
    # workload's shape (config 3's full size runs with --workload statistical)
    stat = (surrogate_eval(1_000_000, 2e13, 14, [1, 2], 0)
            if rank == 0 and not args.no_statistical else None)
    ms = slowest_rank_ms(ms, world, dev)
    K = args.steps
    value = whole_job_rate(tests, world, ms)

    # end to end through the public API with host buffers: every step copies
    # the two beams from pinned host memory, runs, and reads the yield back
    pinned = {k: {kk: v.cpu().pin_memory() for kk, v in D.items()} for k, D in (("a", A), ("b", B))}
    h2d = sum(v.numel() * v.element_size() for D in pinned.values() for v in D.values())
    e2e_ms = []
    for i in range(args.warmup + K):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for key, D in (("a", A), ("b", B)):
            for kk, v in D.items():
                v.copy_(pinned[key][kk], non_blocking=True)
        col.reset_yield()
        graph_run()
        cnt, wsum = col.yield_()  # device -> host read of the result
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = whole_job_rate(tests / K, world,
                               slowest_rank_ms(statistics.mean(e2e_ms), world, dev))

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_src = read_peaks()
    # rooflines of the traversal (HBM: its algorithmic bytes per step), the
    # narrow phase (FP32 ALU: the test prefix's operations) and the dominant
    # build phase, each from the per-phase device times of the step-by-step
    # runs; the dominant one by time is the line's roofline
    n_ab = wl.a.n + wl.b.n
    leaves = sum(r["leaves"] for r in per_step)  # one run
    steps_total = K * nsteps
    builds = 2 * steps_total  # one build per beam and step

    def hbm(phase, algo, launch_ms, note):
        ach = algo / (launch_ms / 1e3) / 1e9
        return {"kernel": phase, "bound": "hbm", "achieved": ach, "peak": peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                "algorithmic_bytes_per_launch": algo, "launch_ms": launch_ms, "unit_of_work": note}

    roofs = {}
    roofs["traverse"] = hbm("traverse", 64.0 * n_ab + 8.0 * leaves / nsteps,
                            phase_ms["traverse"] / steps_total,
                            "one step: node records of both trees once, leaf pairs written")
    ops = NARROW_OPS_PER_TEST * tests / K / nsteps
    nms = phase_ms["narrow"] / steps_total
    roofs["narrow"] = {"kernel": "narrow", "bound": "alu", "unit": "FP32 op/s",
                       "achieved": ops / (nms / 1e3), "peak": FP32_OPS_PEAK,
                       "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz",
                       "frac": ops / (nms / 1e3) / FP32_OPS_PEAK, "launch_ms": nms,
                       "ops_per_test": NARROW_OPS_PER_TEST, "traffic": None}
    for ph in ("sort", "refit", "emit", "propagate"):
        per_unit, _ = algorithmic_bytes(ph, wl.a.n, wl.b.n, None, 0, 0)
        if ph == "sort":  # the unit is one digit pass over one beam
            passes = max(launches[ph] - builds, 1)  # minus one scan per build
            roofs[ph] = hbm(ph, per_unit * n_ab / 2, phase_ms[ph] / passes, "one pass, one beam")
        else:
            roofs[ph] = hbm(ph, per_unit * n_ab / 2, phase_ms[ph] / builds, "one beam's build")
    dom = max(roofs, key=lambda p: phase_ms[p])
    # busy steps: those with at least 5% of the peak step's narrow-phase tests
    peak_tests = max(r["tests"] for r in per_step) if per_step else 0
    busy = [r for r in per_step if peak_tests and r["tests"] >= 0.05 * peak_tests]
    tb = sum(r["traverse"] for r in busy)
    tn = sum(r["narrow"] for r in busy)
    busy_bytes = sum(64.0 * n_ab + 8.0 * r["leaves"] for r in busy)
    busy_ops = NARROW_OPS_PER_TEST * sum(r["tests"] for r in busy)
    roofs["traverse"]["busy_steps"] = {
        "steps": [r["step"] for r in busy], "ms": tb, "algorithmic_bytes": busy_bytes,
        "achieved": busy_bytes / (tb / 1e3) / 1e9 if tb > 0 else None,
        "frac": busy_bytes / (tb / 1e3) / 1e9 / peak if tb > 0 else None,
        "per_step_ms": [round(r["traverse"], 4) for r in busy]}
    roofs["narrow"]["busy_steps"] = {
        "steps": [r["step"] for r in busy], "ms": tn,
        "achieved": busy_ops / (tn / 1e3) if tn > 0 else None,
        "frac": busy_ops / (tn / 1e3) / FP32_OPS_PEAK if tn > 0 else None,
        "per_step_ms": [round(r["narrow"], 4) for r in busy],
        "narrow_tests": [r["tests"] for r in busy]}
    # DRAM traffic from profiles/traffic.txt: the traversal's on busy steps (with
    # the capture's own algorithmic bytes: the leaf-pair count depends on the
    # knobs), the build kernels' per launch like their rooflines
    tr = read_traffic("traverse")
    if tr is not None:
        dram, algo = float(tr["bytes_per_launch"]), float(tr["algorithmic_bytes_per_launch"])
        roofs["traverse"]["busy_steps"]["traffic"] = {
            "steps": tr["steps"], "knobs": tr["knobs"], "dram_bytes_per_launch": dram,
            "algorithmic_bytes_per_launch": algo, "dram_over_algorithmic": dram / algo}
    roofline = dict(roofs[dom])
    td = read_traffic(dom) if dom != "traverse" else None
    roofline["traffic"] = float(td["bytes_per_launch"]) if td is not None else None
    roofline["traffic_note"] = (
        "DRAM bytes were captured on busy steps only (rooflines.traverse.busy_steps.traffic)"
        if dom == "traverse" else
        ("dram__bytes_read.sum + dram__bytes_write.sum per launch, profiles/traffic.txt"
         if td is not None else "not captured for this kernel"))
    cpu = (cpu_baseline(wl, a_np, b_np, first, nsteps)
           if (world == 1 and not args.no_cpu_baseline) else None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": config_of(wl, L2_NOTE, nsteps, first),
        "collided_pairs_per_s": world * hits / (ms / 1e3),
        "all_pairs_per_s": whole_job_rate(wl.a.n * wl.b.n * nsteps * K, world, ms),
        "all_pairs_note": "context only: N_A * N_B * time steps per second, the all-pairs work "
                          "the hierarchy avoids",
        "hits_per_run": hits / K, "narrow_tests_per_run": tests / K, "band_per_run": band / K,
        "node_tests_per_run": work.get("node_tests"), "leaf_pairs_per_run": work.get("leaf_pairs"),
        "path": "trilens_run: all steps of a run as one captured CUDA graph",
        "phase_ms_per_run": {p: phase_ms[p] / K for p in PHASES},
        "phase_source": "the same runs built and collided step by step with CUDA events "
                        "around every phase (after the timed region)",
        "stepwise_ms_per_run": statistics.mean(sw_ms),
        "roofline": roofline,
        "rooflines": roofs,
        "roofline_note": "per-launch averages over every launch of the run (most time steps "
                         "are almost empty: the bunches cross in the first ~10); busy_steps "
                         "gives the steps where they cross",
        "pair_products": pairs,
        "depletion": depl,
        "ip_regime": ipr,
        "crossing90_2x5e7": crossing,
        "statistical_2x1e6_sample": stat,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 16},
        # the graph holds the step-by-step path's kernels plus one status kernel per step
        "gpu_launches": int(sum(launches.values())) + K * nsteps,
        "tuning": tuned,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """The batching workload (not the default line): 256 independent
    instances, 1,024-262,144 photons per beam, 16 steps, one CUDA graph."""
    import torch

    from paper_1608_01125_gb300 import binding
    torch.cuda.set_device(0)
    wls = [synth.batch_instance(i) for i in range(256)]
    A, B = zip(*[synth.beams(w) for w in wls])
    bt = binding.Batch(list(A), list(B), wls[0].dt, wls[0].kappa)
    tuned = bt.autotune([7, 8], os.path.join(ROOT, "paper_1608_01125_gb300",
                                             "_tuning_cache.json")) if args.tune else bt.tuning()
    for _ in range(max(args.warmup, 1)):
        y = bt.run(0, 16)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        y = bt.run(0, 16)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    pairs = sum(len(a["px"]) * len(b["px"]) for a, b in zip(A, B)) * 16
    line = {"metric": "photon-pair tests/s, 256 batched instances", "value": pairs * args.steps / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batch_256", "instances": 256,
                       "photons_per_beam": [min(len(a["px"]) for a in A), max(len(a["px"]) for a in A)],
                       "photons_total_per_side": int(sum(len(a["px"]) for a in A)), "time_steps": 16,
                       "graph": True, "l2": "flushed (256 MiB write) before every timed step"},
            "hits_per_run": float(y[:, 0].sum()), "tuning": tuned}
    print(json.dumps(line), flush=True)
    bt.close()


def surrogate_eval(n, kappa, L, train_seeds, test_seed, taus=(1e30,), epochs=30,
                   model=None):
    """The learned statistical regime on the statistical workload's shape
    (weights U[1,10], Gamma(2, 5 MeV) energies, head-on Gaussian beams,
    32 steps of 20 fs) with n macro-photons per beam: a network trained on
    the draws train_seeds (all steps, level L) estimates the draw test_seed.
    The exact GPU traversal of the same steps, with autotuned knobs, is the
    reference for the yield error and the time; beside the network: the
    paper's ST rate of the same node pairs (no network, no fitted scale) and
    that rate times the one scale fitted on the training pairs.  Device times
    with CUDA events: exact = frontier + traversal + narrow phase + band +
    yield after each step's build; surrogate = cut traversal, features,
    network, estimate and the exact fallback."""
    import torch

    from paper_1608_01125_gb300 import binding
    model = model or os.path.join(tempfile.gettempdir(), f"trilens_surrogate_L{L}_{n}.bin")
    t0 = time.perf_counter()
    wl1 = synth.statistical_1e8(n=n, seed=train_seeds[0])
    a1, b1 = synth.beams(wl1)
    with binding.Collider(a1, b1, wl1.dt, kappa) as col:
        col.surrogate_collect(list(range(wl1.steps)), L)
        for sd in train_seeds[1:]:  # further draws: their labelled pairs join the training set
            wlx = synth.statistical_1e8(n=n, seed=sd)
            ax, bx = synth.beams(wlx)
            with binding.Collider(ax, bx, wlx.dt, kappa) as cx:
                cx.surrogate_collect(list(range(wlx.steps)), L)
                x, lab, st = cx.surrogate_dataset()
            del ax, bx
            col.surrogate_add_samples(x, lab, st, L)
        col.surrogate_fit(epochs, 7)
        info = col.surrogate_info()
        col.surrogate_save(model)
    del a1, b1
    t_train = time.perf_counter() - t0
    wl0 = synth.statistical_1e8(n=n, seed=test_seed)
    a0, b0 = synth.beams(wl0)
    exact = ms_exact = ms_build = 0.0
    acc = {t: dict(sur=0.0, st=0.0, ms=0.0, pairs=0, fb=0) for t in taus}
    with binding.Collider(a0, b0, wl0.dt, kappa) as col:
        trained_knobs = col.tuning()  # the hierarchy the network was trained on
        tuned = col.autotune([wl0.steps // 2 - 1, wl0.steps // 2, wl0.steps // 2 + 1])
        col.timing(True)
        for k in range(wl0.steps):  # the exact traversal with the fastest knobs
            col.phase_ms(reset=True)
            col.build(k)
            col.collide(k)
            ph, _ = col.phase_ms()
            ms_exact += sum(ph[p] for p in ("expand", "traverse", "narrow", "band", "yield"))
            ms_build += sum(ph[p] for p in ("propagate", "sort", "gather", "emit", "refit"))
            exact += col.stats()["weighted"]
        col.set_tuning(*[trained_knobs[k] for k in ("leaf_bucket", "stack_depth", "block_shape",
                                                    "budget")])
        col.surrogate_load(model)
        for k in range(wl0.steps):  # the surrogate on the level-L cut it was trained on
            for t in taus:
                r = col.surrogate_step(k, L, t)
                q = acc[t]
                q["sur"] += r["yield"]
                q["st"] += r["st_yield"]
                q["ms"] += r["ms"]
                q["pairs"] += r["pairs"]
                q["fb"] += r["fallback_pairs"]
        torch.cuda.synchronize()
    out = []
    for t in taus:
        q = acc[t]
        out.append({"tau": t, "speedup": ms_exact / q["ms"], "yield_error": (q["sur"] - exact) / exact,
                    "st_rate_error": (q["st"] - exact) / exact,
                    "st_scaled_error": (info["st_calib"] * q["st"] - exact) / exact,
                    "st_scale": info["st_calib"], "exact_weighted_yield": exact,
                    "surrogate_weighted_yield": q["sur"], "exact_traversal_ms": ms_exact,
                    "surrogate_ms": q["ms"], "build_ms": ms_build, "pairs": q["pairs"],
                    "fallback_pairs": q["fb"]})
    return {"photons_per_beam": n, "kappa": kappa, "level_L": L, "time_steps": wl0.steps,
            "train": f"seeds {list(train_seeds)}, all steps", "test": f"seed {test_seed}, all steps",
            "train_samples": info["samples"], "train_s": t_train, "exact_tuning": tuned,
            "results": out}


def run_statistical(args):
    """The statistical workload (not the default line): 2 x 1e8 macro-photons,
    weights U[1,10], Gamma(2, 5 MeV) energies, 32 steps; see surrogate_eval."""
    import torch
    torch.cuda.set_device(0)
    seeds = [int(x) for x in str(args.train_seeds).split(",")]
    taus = [float(t) for t in str(args.tau).split(",")]
    wl = synth.statistical_1e8(n=args.stat_photons)
    r = surrogate_eval(args.stat_photons, wl.kappa, args.level, seeds, 0, taus)
    for q in r["results"]:
        line = {"metric": "surrogate vs exact GPU traversal speedup at <=1% yield error",
                "value": q["speedup"], "unit": "x", "n_gpus": 1, "steps": wl.steps,
                "warmup": 0, "ms_per_step": q["surrogate_ms"] / wl.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16 network, f32+f64 exact", "data": "synthetic",
                "config": {"workload": wl.name, "photons_per_beam": args.stat_photons,
                           "time_steps": wl.steps, "level_L": args.level, "tau": q["tau"],
                           "train": r["train"], "test": r["test"]},
                **{k: v for k, v in q.items() if k != "tau"},
                "train_samples": r["train_samples"], "train_s": r["train_s"],
                "exact_tuning": r["exact_tuning"]}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-depletion", action="store_true",
                    help="skip the depletion leg (run-long depletion after each step)")
    ap.add_argument("--no-statistical", action="store_true",
                    help="skip the surrogate leg on a 2 x 1e6 statistical sample")
    ap.add_argument("--no-crossing", action="store_true",
                    help="skip the leg on busy steps of the 2 x 5e7 crossing workload")
    ap.add_argument("--no-ip", action="store_true",
                    help="skip the IP-regime leg (swarm split + exact run of real photons)")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the autotuner (default knobs)")
    ap.add_argument("--knobs", default="",
                    help="fixed traversal knobs instead of the autotuner: leaf bucket, stack "
                         "depth, warps per block, budget (comma-separated)")
    ap.add_argument("--photons", type=int, default=1 << 20)
    ap.add_argument("--workload", default="headon_2x1M",
                    choices=("headon_2x1M", "batch256", "statistical"))
    ap.add_argument("--level", type=int, default=14, help="statistical workload: cut level L")
    ap.add_argument("--tau", default="1e30",
                    help="statistical workload: fallback threshold(s) on the predicted std, "
                         "comma-separated")
    ap.add_argument("--stat-photons", type=int, default=100_000_000)
    ap.add_argument("--train-seeds", default="1",
                    help="statistical workload: seeds of the training draws, comma-separated")
    ap.add_argument("--first-step", type=int, default=0,
                    help="first time step of each run (profiling a slice of the run)")
    ap.add_argument("--time-steps", type=int, default=0,
                    help="time steps per run (0: the workload's 64)")
    args = ap.parse_args()
    wl = synth.headon_1m(n=args.photons)
    if args.workload == "batch256":
        run_batch(args)
        return
    if args.workload == "statistical":
        run_statistical(args)
        return
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
