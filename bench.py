#!/usr/bin/env python
"""Benchmark of the GB300 BSP sample sort (one JSON line on stdout, rank 0).

Step = one whole sort (sampling, sample sort, splitter selection, routing,
bucket sort) of the workload below, inputs resident in HBM.  Under torchrun
every rank sorts its own independent instance (the sort shards into
independent problems; no collective is on the data path): weak scaling.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the CPU oracle (the paper's algorithm as an explicit
BSP simulation, single-threaded) on a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import bsp_inputs as gen  # noqa: E402

# The workload the metric is quoted on: 2^28 int32 keys of the paper's uniform
# input [U], p = 4096 buckets, random oversampling with the paper's default
# s = 2 lg^2 n = 1568 (sample 6,422,527 keys), keys only.
WORKLOADS = {
    "uniform_2e28_int32_p4096_random": dict(n=1 << 28, p=4096, sampling=1, s=0, runs=0, pairs=False,
                                           make=lambda n, p, seed: gen.uniform(n, p, seed)),
    "uniform_2e28_int32_p4096_regular": dict(n=1 << 28, p=4096, sampling=0, s=4096, runs=4096, pairs=False,
                                            make=lambda n, p, seed: gen.uniform(n, p, seed)),
    "zipf_2e28_int32_pairs_p4096_regular": dict(n=1 << 28, p=4096, sampling=0, s=4096, runs=4096, pairs=True,
                                               block_sort_kernel="run_sample_lowcard_kernel",
                                               make=lambda n, p, seed: gen.zipf(n, seed=seed)),
    # the regular configurations ended by the paper's merge (Fig. 1 steps 9-12),
    # with the bucket-sort final step timed beside them on the same inputs
    "uniform_2e28_int32_p4096_regular_merge": dict(n=1 << 28, p=4096, sampling=0, s=4096, runs=4096,
                                                  pairs=False, final_step=1, compare="sort",
                                                  make=lambda n, p, seed: gen.uniform(n, p, seed)),
    "zipf_2e28_int32_pairs_p4096_regular_merge": dict(n=1 << 28, p=4096, sampling=0, s=4096, runs=4096,
                                                     pairs=True, final_step=1, compare="sort",
                                                     block_sort_kernel="run_sample_lowcard_kernel",
                                                     make=lambda n, p, seed: gen.zipf(n, seed=seed)),
    # the merge's kernels on a quarter of the data (16-key segments as at 2^28),
    # for full ncu captures
    "uniform_2e26_int32_p2048_regular_merge": dict(n=1 << 26, p=2048, sampling=0, s=2048, runs=2048,
                                                  pairs=False, final_step=1,
                                                  make=lambda n, p, seed: gen.uniform(n, p, seed)),
    # the cost of the duplicate handling (Sec. 6.4 measures it): the headline
    # sort without the tie-break, and with it (timed beside) on the same keys
    "uniform_2e28_int32_p4096_random_nodup": dict(n=1 << 28, p=4096, sampling=1, s=0, runs=0, pairs=False,
                                                 duplicates=1, compare="tags",
                                                 make=lambda n, p, seed: gen.uniform(n, p, seed)),
    # the 2^28 workload's kernels on a quarter of the data, for full ncu
    # captures (inputs still larger than L2)
    "uniform_2e26_int32_p4096_random": dict(n=1 << 26, p=4096, sampling=1, s=0, runs=0, pairs=False,
                                           make=lambda n, p, seed: gen.uniform(n, p, seed)),
    # the 2^28 workload's bucket shape (65,536-key buckets on clusters of 8,
    # count sorts in the occupancy-mask regime) on half the data, for full ncu
    # captures of the bucket sort
    "uniform_2e27_int32_p2048_random": dict(n=1 << 27, p=2048, sampling=1, s=0, runs=0, pairs=False,
                                           make=lambda n, p, seed: gen.uniform(n, p, seed)),
    # the 2^28 workload's buckets exactly (65,536 keys spanning 2^19 values,
    # clusters of 8) on half the data: keys uniform on [0, 2^30), p = 2048
    "uniform30_2e27_int32_p2048_random": dict(n=1 << 27, p=2048, sampling=1, s=0, runs=0, pairs=False,
                                             make=lambda n, p, seed: gen.uniform(n, p, seed) >> 1),
    # the Zipf pairs configuration on a quarter of the data, for full ncu
    # captures of its kernels
    "zipf_2e26_int32_pairs_p4096_regular": dict(n=1 << 26, p=4096, sampling=0, s=4096, runs=4096, pairs=True,
                                               make=lambda n, p, seed: gen.zipf(n, seed=seed)),
    # the randomized config's shape: 2^26 keys, p = 1024
    "uniform_2e26_int32_p1024_random": dict(n=1 << 26, p=1024, sampling=1, s=0, runs=0, pairs=False,
                                           make=lambda n, p, seed: gen.uniform(n, p, seed)),
    # learned classifier against the splitter tree: 2^28 float64 keys of an
    # 8-component Gaussian mixture (Dirichlet(0.3) weights), p = 4096, s = 16
    # (both classifiers with the same plan: two sub-buckets per bucket)
    "gmm_2e28_f64_p4096_random_learned": dict(n=1 << 28, p=4096, sampling=1, s=16, runs=0, pairs=False,
                                             dtype="f64", classify=1, compare="tree", refine=2,
                                             make=lambda n, p, seed: gen.gmm(n, seed=seed)),
    # the same on a quarter of the data, for ncu captures of the two routings
    "gmm_2e26_f64_p4096_random_learned": dict(n=1 << 26, p=4096, sampling=1, s=16, runs=0, pairs=False,
                                             dtype="f64", classify=1, compare="tree", refine=1,
                                             make=lambda n, p, seed: gen.gmm(n, seed=seed)),
    # batched: 20,000 int32 instances, sizes log-uniform on [2^8, 2^22],
    # alternately uniform [U] and Zipf(1.1) over 256 values; the first
    # instances up to 2^28 keys in all, or all 20,000 (about 2^33 keys)
    "batched_20000_int32_first_2e28": dict(kind="batched", count=20000, cap=1 << 28, p=0, sampling=1),
    "batched_20000_int32_all": dict(kind="batched", count=20000, cap=None, p=0, sampling=1),
}
DEFAULT_WORKLOAD = "uniform_2e28_int32_p4096_random"
METRIC = "keys/sec and % HBM roofline, 2^28 int32; learned/batched vs plain, bit-exact"

# Algorithmic bytes per key of each timed phase (keys only, 4-byte keys): the
# routing pass reads every key and writes it once (8 B); the bucket sort reads
# and writes every key once (8 B).  With 4-byte payloads both double.
PHASES = ["sample", "sample_sort", "splitters", "route", "bucket_sort"]
PHASE_KERNEL = {("route", False): "route_keys_kernel", ("bucket_sort", False): "bucket_keys32_kernel",
                ("route", True): "route_kernel", ("bucket_sort", True): "bucket_sort_kernel"}
PHASE_KERNEL_F64 = {"bucket_sort": "bucket_keys_kernel"}
# the variant timed beside a workload: (label, the parameters that change)
COMPARE = {"tree": ("tree", dict(classify=0)), "sort": ("bucket_sort_final_step", dict(final_step=0)),
           "tags": ("with_duplicate_handling", dict(duplicates=0))}

# dram__bytes_read.sum + dram__bytes_write.sum per key of each kernel from one
# ncu capture (its summary is under profiles/), valid while the kernel source is unchanged:
# routing from the 2^26-key capture (4096 buckets, as at 2^28), the bucket sort
# from the 2^27-key capture on [0, 2^30) (65,536-key buckets spanning 2^19
# values on clusters of 8, as at 2^28);
# both kernels stream every key once, so bytes per key carry over to 2^28
# (bytes per key, source hash, payloads) of each capture; the segment copy's
# from the 2^26-pair Zipf capture (4096 buckets of 16-key segments, as at 2^28)
NCU_TRAFFIC = {"route_keys_kernel": ((271.608576e6 + 223.674880e6) / (1 << 26), "8baca4c618da453f", False),
               "bucket_keys32_kernel": ((537.268992e6 + 486.783232e6) / (1 << 27), "b2f4fe6e7d92e3af", False),
               "segment_copy_kernel": ((617.909248e6 + 494.979328e6) / (1 << 26), "333c4e171f9cd65e", True)}
KERNEL_SOURCE = {"route_kernel": ["paper_1408_6729_gb300/csrc/route.cu"],
                 "segment_copy_kernel": ["paper_1408_6729_gb300/csrc/merge.cu"],
                 "route_keys_kernel": ["paper_1408_6729_gb300/csrc/route_keys.cu",
                                       "paper_1408_6729_gb300/csrc/classify.cuh",
                                       "paper_1408_6729_gb300/csrc/kernels.cuh"],
                 "bucket_sort_kernel": ["paper_1408_6729_gb300/csrc/bucket.cu",
                                        "paper_1408_6729_gb300/csrc/segsort.cuh"],
                 "bucket_keys_kernel": ["paper_1408_6729_gb300/csrc/bucket.cu",
                                        "paper_1408_6729_gb300/csrc/segsort_keys.cuh"],
                 "bucket_keys32_kernel": ["paper_1408_6729_gb300/csrc/bucket.cu",
                                          "paper_1408_6729_gb300/csrc/bucket_keys32.cuh",
                                          "paper_1408_6729_gb300/csrc/segsort_keys.cuh",
                                          "paper_1408_6729_gb300/csrc/radix.cuh"]}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 50 ms (one streaming
    nvidia-smi process) from the start of the warm-up to the end of the timed
    region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self._t = None

    def _read(self):
        for line in self.proc.stdout:
            line = line.strip()
            if line:
                self.rows.append([x.strip() for x in line.split(",")])

    def __enter__(self):
        if self.proc is not None:  # already sampling (started before the warm-up)
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)  # the first sample arrives before the work starts
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=10)
            except Exception:
                self.proc.kill()
            self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "window": "warm-up and timed region"}


def source_hash(paths):
    h = hashlib.sha256()
    for path in paths:
        h.update(open(os.path.join(ROOT, path), "rb").read())
    return h.hexdigest()[:16]


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    return world, rank, local, pg


def max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


# ------------------------------------------------------------------ CPU oracle arm

def host_threads():
    return max(1, os.cpu_count() or 1)


def oracle_rate(wl, budget_s=12.0, seed=1, threads=1):
    """Oracle keys/s on a bounded sample of the workload: same generator, p, s,
    runs and mode; n doubles from 2^20 until one sort takes budget_s/4."""
    import oracle
    oracle.build()
    n = 1 << 20
    while True:
        keys = wl["make"](n, wl["p"], seed)
        vals = np.arange(n, dtype=np.uint32) if wl["pairs"] else None
        t0 = time.perf_counter()
        oracle.sort(keys, wl["p"], wl["s"], wl["runs"], wl["sampling"], seed=seed, vals=vals, want_sample=False,
                    threads=threads, duplicates=wl.get("duplicates", 0))
        t = time.perf_counter() - t0
        if t > budget_s / 4 or n >= wl["n"]:
            return n / t, n, wl["s"], wl["runs"], t
        n *= 2


def cpu_baselines(wl, p):
    """The oracle on all host cores (one thread per group of virtual
    processors, a barrier per superstep) and on one core, and std::sort /
    std::stable_sort on one core, each on a bounded sample of the workload."""
    import oracle
    T = host_threads()
    rate, ns, s_used, runs_used, t_used = oracle_rate(wl, threads=T)
    rate1, ns1, _, _, t1 = oracle_rate(wl, budget_s=8.0, threads=1)
    keys = wl["make"](ns1, wl["p"], 1)
    std = {}
    for stable in (False, True):
        t0 = time.perf_counter()
        oracle.std_sort(keys, stable=stable)
        std["std_stable_sort" if stable else "std_sort"] = ns1 / (time.perf_counter() - t0)
    return {"value": rate, "unit": "keys/s", "cores": T, "kind": "oracle",
            "sample": f"{ns} keys of the same generator, p={p}, s={s_used}, runs={runs_used or p}, "
                      f"{t_used:.1f} s on {T} threads",
            "oracle_1_thread": {"value": rate1, "sample": f"{ns1} keys, {t1:.1f} s"},
            "std_sort_1_thread": {"value": std["std_sort"], "sample": f"{ns1} keys (keys only)"},
            "std_stable_sort_1_thread": {"value": std["std_stable_sort"], "sample": f"{ns1} keys (keys only)"},
            "cpu": cpu_model()}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu part"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def run_reference(args, wl, name):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    T = host_threads()
    rate, n, s, runs, t = oracle_rate(wl, budget_s=min(12.0, 150.0 / max(1, args.steps + args.warmup)), threads=T)
    times = []
    import oracle
    keys = wl["make"](n, wl["p"], 1)
    vals = np.arange(n, dtype=np.uint32) if wl["pairs"] else None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.sort(keys, wl["p"], s, runs, wl["sampling"], seed=1, vals=vals, want_sample=False, threads=T,
                    duplicates=wl.get("duplicates", 0))
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = n * len(times) / tot
    sample = (f"{n} keys of the workload's generator, p={wl['p']}, s={s}, runs={runs or wl['p']}, "
              f"one oracle sort per step on {T} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if wl.get("dtype") == "f64" else "int32",
            "data": "synthetic", "config": {"workload": name, "n": wl["n"], "p": wl["p"]},
            "cpu_baseline": {"value": value, "unit": "keys/s", "cores": T, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_gpu(args, wl, name):
    import torch
    import paper_1408_6729_gb300 as bsps
    from paper_1408_6729_gb300 import build as lib_build

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        lib_build.build()
    barrier(pg)
    lib_build.build()  # no-op once built
    n, p = wl["n"], wl["p"]
    f64 = wl.get("dtype") == "f64"
    code = bsps.BSPS_F64 if f64 else bsps.BSPS_I32
    prm = params_of(bsps, wl, args, 1 + rank)
    plan = bsps.bsps_get_plan(n, code, prm, wl["pairs"])
    keys_h = np.ascontiguousarray(wl["make"](n, p, 1 + rank))
    kin = torch.from_numpy(keys_h).to(dev)
    kout = torch.empty_like(kin)
    vin = vout = None
    if wl["pairs"]:
        vin = torch.arange(n, dtype=torch.int32, device=dev)
        vout = torch.empty_like(vin)
    sizes = torch.empty(p, dtype=torch.int64, device=dev)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    # one set of phase events per timed step, created (recorded once) up front
    step_events = [[torch.cuda.Event(enable_timing=True) for _ in range(bsps.BSPS_PHASES)]
                   for _ in range(args.steps)]
    for evs in step_events:
        for e in evs:
            e.record(stream)
    torch.cuda.synchronize()
    launches = ctypes.c_int32(0)

    def step(timed_events=None, count=None):
        rc = bsps.bsps_sort_debug(kin, vin, kout, vout, n, code, prm, sizes, ws, phase_events=timed_events,
                                  launches=count)
        if rc:
            raise RuntimeError(bsps.bsps_strerror(rc))

    def sort_into(src, dst):
        # the public entry point a user calls, on the current stream
        if vin is None:
            rc = bsps.bsps_sort_keys(src, dst, n, code, prm, sizes, ws)
        else:
            rc = bsps.bsps_sort_pairs(src, vin, dst, vout, n, code, prm, sizes, ws)
        if rc:
            raise RuntimeError(bsps.bsps_strerror(rc))

    clk = ClockSampler(local).__enter__()
    for _ in range(args.warmup):
        step()
    st = bsps.bsps_read_stats(ws)
    if st.status:
        raise RuntimeError(f"device status {bsps.bsps_strerror(st.status)}")

    # timed region: K whole sorts, back to back on one stream
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_launches = 0
    with clk:
        barrier(pg)
        torch.cuda.synchronize()
        start.record(stream)
        for k in range(args.steps):
            step(step_events[k], launches)
            total_launches += launches.value
        end.record(stream)
        torch.cuda.synchronize()
        barrier(pg)
    elapsed_ms = start.elapsed_time(end)
    phase_ms = {k: sum(evs[i].elapsed_time(evs[i + 1]) for evs in step_events) for i, k in enumerate(PHASES)}
    elapsed_ms = max_over_ranks(pg, elapsed_ms)
    st = bsps.bsps_read_stats(ws)
    if st.status:
        raise RuntimeError(f"device status {bsps.bsps_strerror(st.status)}")
    # the last output, after the timed region: equal to the input sorted by
    # torch, and its bucket sizes equal to the oracle's (same keys and seed)
    if not torch.equal(torch.sort(kin).values, kout):
        raise RuntimeError("output differs from the sorted input")
    verified = None
    if not args.no_verify and rank == 0:
        import oracle
        t0 = time.perf_counter()
        ref = oracle.sort(keys_h, p, wl["s"], wl["runs"], wl["sampling"], seed=prm.seed, want_sample=False,
                          vals=np.arange(n, dtype=np.uint32) if wl["pairs"] else None, threads=host_threads(),
                          duplicates=wl.get("duplicates", 0))
        if not np.array_equal(sizes.cpu().numpy(), ref.bucket_sizes):
            raise RuntimeError("bucket sizes differ from the oracle's")
        if wl["pairs"] and not np.array_equal(vout.cpu().numpy().view(np.uint32), ref.vals):
            raise RuntimeError("payloads differ from the oracle's")
        verified = {"sorted_equals_torch_sort": True, "bucket_sizes_equal_oracle": True,
                    "payloads_equal_oracle": True if wl["pairs"] else None,
                    "oracle_s": round(time.perf_counter() - t0, 1)}
        del ref
    compare = None
    if wl.get("compare") and not args.no_compare:
        compare = compare_variant(args, bsps, kin, vin, kout, vout, sizes, n, code, wl, rank, st, stream,
                                  elapsed_ms)

    # end to end through the C ABI with host buffers: H2D of the keys, the sort,
    # D2H of the sorted keys, every step
    if args.no_e2e:
        e2e_ms, e2e_steps = float("nan"), 0
    else:
        e2e_ms, e2e_steps = run_e2e(args, stream, kin, kout, keys_h, sort_into, pg, n)
    if rank != 0:
        return
    return report(args, wl, name, world, n, p, plan, st, per_step_of(phase_ms, args), elapsed_ms, e2e_ms,
                  e2e_steps, total_launches, clk, compare, verified)


def params_of(bsps, wl, args, seed, **override):
    kw = dict(s=wl["s"], runs=wl["runs"], sampling=wl["sampling"], seed=seed,
              refine=args.refine or wl.get("refine", 0), classify=wl.get("classify", 0),
              final_step=wl.get("final_step", 0), duplicates=wl.get("duplicates", 0))
    kw.update(override)
    return bsps.make_params(wl["p"], **kw)


def compare_variant(args, bsps, kin, vin, kout, vout, sizes, n, code, wl, rank, st_this, stream, this_ms):
    """The same sort with the variant COMPARE names (the splitter tree, the
    bucket-sort final step, the duplicate handling): time, and identical
    sorted output (and bucket sizes, except without the tie-break)."""
    import torch
    label, override = COMPARE[wl["compare"]]
    prm = params_of(bsps, wl, args, 1 + rank, **override)
    plan = bsps.bsps_get_plan(n, code, prm, vin is not None)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=kin.device)
    out = torch.empty_like(kout)
    vo = torch.empty_like(vout) if vin is not None else None
    sz = torch.empty_like(sizes)

    def one():
        if vin is None:
            assert bsps.bsps_sort_keys(kin, out, n, code, prm, sz, ws) == 0
        else:
            assert bsps.bsps_sort_pairs(kin, vin, out, vo, n, code, prm, sz, ws) == 0
    for _ in range(args.warmup):
        one()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    if bsps.bsps_read_stats(ws).status:
        raise RuntimeError("the compared variant reported an error")
    other_ms = e0.elapsed_time(e1) / args.steps
    as_bits = (lambda t: t.view(torch.int64)) if code == bsps.BSPS_F64 else (lambda t: t)
    same = bool(torch.equal(as_bits(out), as_bits(kout)))
    if vin is not None:
        same = same and bool(torch.equal(vo, vout))
    same_sizes = bool(torch.equal(sz, sizes))
    this = "learned" if wl["compare"] == "tree" else "this"
    res = {"other": label, f"{label}_ms_per_step": other_ms, f"{this}_ms_per_step": this_ms / args.steps,
           f"{this}_vs_{label}": other_ms / (this_ms / args.steps), "identical_output": same,
           "identical_bucket_sizes": same_sizes}
    if wl["compare"] == "tree":
        res["mispredicted_frac"] = st_this.mispredicted / n
        res["correction_steps_per_key"] = st_this.correction_steps / n
    return res


def per_step_of(phase_ms, args):
    return {k: v / args.steps for k, v in phase_ms.items()}


def run_e2e(args, stream, kin, kout, keys_h, step, pg, n):
    """Sorts through the C ABI from and to pinned host buffers: every step
    copies its keys in, sorts them and copies the sorted keys out.  Steps are
    pipelined over three streams (the copy of step i+1's keys in and of step
    i's result out overlap the sort of another step; device buffers are
    double-buffered)."""
    import torch
    dev = kin.device
    h_in = torch.from_numpy(keys_h).pin_memory()
    h_out = [torch.empty_like(h_in).pin_memory() for _ in range(2)]
    d_in = [kin, torch.empty_like(kin)]
    d_out = [kout, torch.empty_like(kout)]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    e2e_steps = max(2, min(args.steps, 10))

    def pipeline(steps):
        in_ready = [torch.cuda.Event() for _ in range(steps)]
        sorted_ = [torch.cuda.Event() for _ in range(steps)]
        out_done = [torch.cuda.Event() for _ in range(steps)]
        for i in range(steps):
            b = i % 2
            with torch.cuda.stream(s_in):
                if i >= 2:
                    s_in.wait_event(sorted_[i - 2])  # d_in[b] is free again
                d_in[b].copy_(h_in, non_blocking=True)
                in_ready[i].record(s_in)
            stream.wait_event(in_ready[i])
            if i >= 2:
                stream.wait_event(out_done[i - 2])  # d_out[b] is free again
            step(d_in[b], d_out[b])
            sorted_[i].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(sorted_[i])
                h_out[b].copy_(d_out[b], non_blocking=True)
                out_done[i].record(s_out)
        stream.wait_event(out_done[steps - 1])
        if steps > 1:
            stream.wait_event(out_done[steps - 2])

    pipeline(2)
    torch.cuda.synchronize()
    barrier(pg)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_in.wait_event(e0)
    pipeline(e2e_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(pg, e0.elapsed_time(e1))
    last = h_out[(e2e_steps - 1) % 2].numpy()
    ref = kout.cpu().numpy() if (e2e_steps - 1) % 2 == 0 else d_out[1].cpu().numpy()
    assert np.array_equal(last[:: max(1, n // 4096)], ref[:: max(1, n // 4096)])
    return e2e_ms, e2e_steps


def report(args, wl, name, world, n, p, plan, st, per_step, elapsed_ms, e2e_ms, e2e_steps, total_launches, clk,
           compare=None, verified=None):
    pk, pk_kind = peaks()
    key_bytes = 8 if wl.get("dtype") == "f64" else 4
    kb = key_bytes + (4 if wl["pairs"] else 0)
    merge = wl.get("final_step", 0) == 1
    # regular sampling of 4-byte keys keeps the sorted blocks and routes by
    # their partition and segment copies (Fig. 1 steps 9-11)
    keep = wl["sampling"] == 0 and key_bytes == 4 and not wl.get("classify")
    # (kernel, algorithmic bytes) of every phase that moves all the keys
    model = {}
    if wl["sampling"] == 0:  # the block sort reads every key (and writes the sorted blocks when it keeps them)
        # keys without payloads in whole 16-byte groups: the counting sort (and the tag kernel)
        counting = keep and not wl["pairs"] and n % 4 == 0 and -(-n // plan.R) % 4 == 0
        kern0 = "run_sample_count_kernel" if counting else "run_sample_keys_kernel"
        model["sample"] = (wl.get("block_sort_kernel", kern0), n * (2 * kb if keep else key_bytes))
    if merge:
        model["bucket_sort"] = ("merge_bucket_kernel", n * 2 * kb)
    else:
        for ph in ("route", "bucket_sort"):
            kern = PHASE_KERNEL[(ph, bool(wl["pairs"]))]
            if key_bytes == 8 and not wl["pairs"]:
                kern = PHASE_KERNEL_F64.get(ph, kern)
            if ph == "route" and keep:
                kern = "segment_copy_kernel"
            model[ph] = (kern, n * 2 * kb)
    dom = max(model, key=lambda k: per_step[k])
    kern, alg_bytes = model[dom]
    achieved = alg_bytes / (per_step[dom] * 1e-3) / 1e9
    traffic = None
    if kern in NCU_TRAFFIC and NCU_TRAFFIC[kern][1] == source_hash(KERNEL_SOURCE[kern]) and \
            wl.get("dtype") != "f64" and bool(wl["pairs"]) == NCU_TRAFFIC[kern][2]:
        traffic = NCU_TRAFFIC[kern][0] * n
    ms_step = elapsed_ms / args.steps
    value = world * n / (ms_step * 1e-3)
    rec = 8 if key_bytes == 4 else 16
    b_alg = 4 * kb + plan.sample_size * (key_bytes + 2 * rec) / n + \
        (key_bytes if wl["sampling"] == 0 and not merge else 0)
    cpu = None
    if world == 1 and not args.no_baseline and wl.get("dtype") != "f64":
        cpu = cpu_baselines(wl, p)
    line = {
        "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if key_bytes == 8 else "int32", "data": "synthetic",
        "config": {"workload": name, "n": n, "p": p, "sampling": "random" if wl["sampling"] else "regular",
                   "s": plan.s, "runs": plan.R, "sample_size": plan.sample_size, "pairs": wl["pairs"],
                   "refine": plan.refine, "bucket_cluster": plan.bucket_cluster,
                   "classify": "learned" if wl.get("classify") else "tree",
                   "final_step": "merge" if merge else "bucket_sort",
                   "duplicate_handling": not wl.get("duplicates", 0),
                   "l2": "inputs (1 GiB) larger than L2 (126 MB); no flush",
                   "parallelism": f"independent sorts x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": traffic, "kernel": kern,
                     "peak_source": f"{pk_kind} hbm_gbs", "alg_bytes_per_launch": alg_bytes},
        "path_roofline": {"alg_bytes_per_key": b_alg,
                          "frac": n * b_alg / (ms_step * 1e-3) / 1e9 / pk["hbm_gbs"]},
        "phases_ms": per_step,
        "cpu_baseline": cpu,
        "e2e": None if args.no_e2e else {"value": world * n * e2e_steps / (e2e_ms * 1e-3), "unit": "keys/s",
                                         "h2d_bytes_per_step": n * key_bytes, "d2h_bytes_per_step": n * key_bytes,
                                         "ms_per_step": e2e_ms / e2e_steps, "steps": e2e_steps,
                                         "how": "bsps_sort_keys on keys copied in from pinned host memory, "
                                                "sorted keys copied out; copies of neighbouring steps overlap "
                                                "the sort (3 streams, double-buffered)"},
        "gpu_launches": total_launches,
        "clocks": clk.summary(),
        "stats": {"max_bucket": st.max_bucket, "max_vbucket": st.max_vbucket, "slow_buckets": st.slow_buckets,
                  "imbalance": st.max_bucket / (n / p) - 1},
    }
    if compare is not None:
        line["learned_vs_tree" if wl["compare"] == "tree" else "compare"] = compare
    if verified is not None:
        line["verified"] = verified
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched arm

def batched_keys(sizes, seed, dev):
    """Instance i's keys: uniform [U] on [0, 2^31) for even i, Zipf(1.1) over
    256 values for odd i, generated on the device in chunks."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    total = int(sizes.sum())
    keys = torch.empty(total, dtype=torch.int32, device=dev)
    table = torch.from_numpy(gen.zipf_values(256)).to(dev)
    w = torch.arange(1, 257, dtype=torch.float64, device=dev) ** -1.1
    cdf = torch.cumsum(w / w.sum(), 0)
    cdf[-1] = 1.0
    off, i0 = 0, 0
    while i0 < len(sizes):
        i1, m = i0, 0
        while i1 < len(sizes) and (m == 0 or m + sizes[i1] <= (1 << 27)):
            m += int(sizes[i1])
            i1 += 1
        parity = torch.from_numpy((np.arange(i0, i1) % 2).astype(np.int32)).to(dev)
        odd = torch.repeat_interleave(parity, torch.from_numpy(sizes[i0:i1]).to(dev)).bool()
        u = torch.randint(0, 2**31 - 1, (m,), generator=g, device=dev, dtype=torch.int64).to(torch.int32)
        r = torch.searchsorted(cdf, torch.rand(m, generator=g, device=dev, dtype=torch.float64), right=True)
        keys[off:off + m] = torch.where(odd, table[r.clamp_(max=255)], u)
        off += m
        i0 = i1
    return keys


def run_batched(args, wl, name):
    import torch
    import paper_1408_6729_gb300 as bsps
    from paper_1408_6729_gb300 import build as lib_build

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        lib_build.build()
    barrier(pg)
    lib_build.build()
    sizes = gen.batched_sizes(wl["count"], 8.0, 22.0, seed=1 + rank)
    if wl["cap"] is not None:
        keep = int(np.searchsorted(np.cumsum(sizes), wl["cap"], side="right"))
        sizes = sizes[:max(1, keep)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    num, total = len(sizes), int(off[-1])
    code = bsps.BSPS_I32
    prm = bsps.make_params(1, sampling=wl["sampling"], seed=1 + rank)
    stream = torch.cuda.current_stream()
    # the autotuner's table (learned classifier from 2^18 keys up)
    tune = bsps.bsps_tune_default()
    tune.learned_min_log2 = 18
    t0 = time.perf_counter()
    tws = torch.empty(bsps.bsps_autotune_workspace_size(code, prm, 22), dtype=torch.uint8, device=dev)
    rc = bsps.bsps_autotune_batched(code, prm, 22, tune, tws)
    if rc:
        raise RuntimeError(f"autotune: {bsps.bsps_strerror(rc)}")
    del tws
    tune_s = time.perf_counter() - t0
    kin = batched_keys(sizes, 1 + rank, dev)
    kout = torch.empty_like(kin)
    base = bsps.bsps_batch_bucket_base(off, tune)
    bsz = torch.empty(max(1, base[-1]), dtype=torch.int64, device=dev)
    ws = torch.empty(bsps.bsps_batch_workspace_size(off, code, prm, tune), dtype=torch.uint8, device=dev)
    offl = off.tolist()

    def step():
        rc = bsps.bsps_sort_batched(kin, kout, offl, code, prm, tune, bsz, ws)
        if rc:
            raise RuntimeError(bsps.bsps_strerror(rc))

    t0 = time.perf_counter()
    step()  # records the graph
    torch.cuda.synchronize()
    record_s = time.perf_counter() - t0
    clk = ClockSampler(local).__enter__()
    for _ in range(args.warmup):
        step()
    st = bsps.bsps_read_stats(ws)
    if st.status:
        raise RuntimeError(f"device status {bsps.bsps_strerror(st.status)}")
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clk:
        barrier(pg)
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(args.steps):
            step()
        end.record(stream)
        torch.cuda.synchronize()
        barrier(pg)
    ms_step = max_over_ranks(pg, start.elapsed_time(end)) / args.steps
    st = bsps.bsps_read_stats(ws)
    if st.status:
        raise RuntimeError(f"device status {bsps.bsps_strerror(st.status)}")

    # the same instances as a loop of single-instance calls (identical output)
    pws = torch.empty(max(bsps.bsps_workspace_size(int(sizes.max()), code,
                                                   bsps.make_params(tune.p[c], sampling=wl["sampling"]))
                          for c in range(8, 23)), dtype=torch.uint8, device=dev)
    lout = torch.empty_like(kin)
    lsz = torch.empty_like(bsz)
    params = []
    for i in range(num):
        n = int(sizes[i])
        c = 0
        while (1 << c) < n:
            c += 1
        c = min(c, 31)
        q = bsps.make_params(tune.p[c], sampling=wl["sampling"], seed=prm.seed + i,
                             classify=1 if (tune.learned_min_log2 > 0 and c >= tune.learned_min_log2) else 0)
        params.append(q)
        need = bsps.bsps_workspace_size(n, code, q)
        if need > pws.numel():
            pws = torch.empty(need, dtype=torch.uint8, device=dev)

    def loop():
        for i in range(num):
            a, b = offl[i], offl[i + 1]
            rc = bsps.bsps_sort_keys(kin[a:] if b > a else None, lout[a:] if b > a else None, b - a, code,
                                     params[i], lsz[base[i]:], pws)
            if rc:
                raise RuntimeError(bsps.bsps_strerror(rc))

    loop()
    torch.cuda.synchronize()
    l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    l0.record(stream)
    loop()
    l1.record(stream)
    torch.cuda.synchronize()
    loop_ms = l0.elapsed_time(l1)
    identical = bool(torch.equal(lout, kout)) and bool(torch.equal(lsz, bsz))
    if not identical:
        raise RuntimeError("batched output differs from the loop of single calls")
    if rank != 0:
        return
    pk, pk_kind = peaks()
    value = world * total / (ms_step * 1e-3)
    alg = 16.0 * total
    line = {
        "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": name, "instances": num, "keys": total, "sizes": "log-uniform [2^8, 2^22]",
                   "mix": "uniform / Zipf(1.1) alternating", "sampling": "random",
                   "on_chip_max_log2": tune.small_max_log2, "learned_min_log2": tune.learned_min_log2,
                   "lanes": tune.lanes, "p_by_class": {c: tune.p[c] for c in range(8, 23)},
                   "l2": "inputs larger than L2; no flush"},
        "roofline": {"bound": "hbm", "achieved": alg / (ms_step * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": alg / (ms_step * 1e-3) / 1e9 / pk["hbm_gbs"], "traffic": None,
                     "kernel": "whole batched call (16 B/key: route and bucket sort read and write each key)",
                     "peak_source": f"{pk_kind} hbm_gbs"},
        "batched_vs_plain_loop": {"loop_ms": loop_ms, "batched_ms": ms_step, "speedup": loop_ms / ms_step,
                                  "identical_output": identical},
        "autotune_s": tune_s, "graph_record_s": record_s,
        "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk.summary(),
        "stats": {"max_bucket": st.max_bucket, "slow_buckets": st.slow_buckets, "mispredicted": st.mispredicted},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle leg (profiling runs)")
    ap.add_argument("--refine", type=int, default=0, help="sub-buckets per bucket (0: the library's choice)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--no-compare", action="store_true", help="skip the variant timed beside (profiling runs)")
    ap.add_argument("--no-verify", action="store_true",
                    help="skip the oracle comparison of the last output (profiling runs)")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        if wl.get("kind") == "batched":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single sorts only"}))
            return
        run_reference(args, wl, args.workload)
    elif wl.get("kind") == "batched":
        run_batched(args, wl, args.workload)
    else:
        run_gpu(args, wl, args.workload)


if __name__ == "__main__":
    main()
