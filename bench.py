"""Benchmark of batched accurate normalization (arXiv 1606.06508) on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras] [--count C]

One step = one call of the library on the whole per-GPU workload: 2^26
binary32 quaternions (1 GiB in, 1 GiB out), normalized with the scaling
algorithm (Algorithm 7) -- the workload the headline metric is quoted on.
Inputs are resident in HBM when the timed region starts and larger than L2,
so no flush is needed between steps.  Rank 0 prints one JSON line with the
whole-job throughput (vectors/s), the roofline of the dominant kernel
(achieved algorithmic bytes per launch over its event-timed duration, against
the measured HBM copy bandwidth), the oracle timed on the host cores on a
bounded sample (cpu_baseline), an end-to-end figure through host buffers
(e2e), the SM clocks sampled during the timed region, and a parity check of
sampled outputs against the oracle.  With N > 1 (torchrun) each rank
normalizes its own batch (weak scaling, no data exchange); the timing is the
max over ranks.

--impl reference times the oracle (plain single-threaded C, run on all host
cores over contiguous ranges) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "normalized vectors/s & HBM GB/s (% peak), fwd and fwd+bwd, 0-ulp vs oracle"
QUAT_COUNT = 1 << 26
QUAT_BYTES = 32  # 16 B read + 16 B written per quaternion
WORKLOAD = "2^26 binary32 quaternions (float4 AoS), forward: Algorithm 7, 50/50 wide-exponent/N(0,1) components"
KERNEL = "k_small_vec16<float,4>"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s, profiling recipe)"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1606_06508_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        e = d.get(kernel)
        if e and e.get("source_hash") == kernel_source_hash():
            return e["dram_bytes_per_launch"], e.get("note")
    except Exception:
        pass
    return None, None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu=timestamp,{self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        self.marks.append(time.time())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        t0, t1 = (self.marks[0], self.marks[-1]) if len(self.marks) >= 2 else (0, math.inf)
        rows = [l for (t, l) in self.lines if t0 <= t <= t1]
        window = "timed region"
        if len(rows) < 3:  # a short timed region: take the warm-up and timed samples together
            rows = [l for (_, l) in self.lines]
            window = "warm-up and timed region"
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in rows:
            parts = [p.strip() for p in l.split(",")]
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    from paper_1606_06508_gb300 import synth
    oracle.build()
    threads = cpu_threads()
    sample = 1 << 17
    x = synth.quaternions_f32(sample, seed=1)
    for _ in range(args.warmup):
        oracle.normalize_threads(x.reshape(-1), dim=4, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.normalize_threads(x.reshape(-1), dim=4, threads=threads)
    dt = time.perf_counter() - t0
    v = args.steps * sample / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "vectors/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_step": f"{sample} quaternions of the same recipe (bounded sample)"},
        "cpu_baseline": {"value": v, "unit": "vectors/s", "cores": threads, "kind": "oracle",
                         "sample": f"{sample} quaternions per step, oracle on {threads} host threads over contiguous ranges"},
        "e2e": {"value": v, "unit": "vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- our arm
def time_events(fn, iters, stream):
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(iters)]
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def cpu_baseline_quat():
    """The oracle on the host cores on a bounded sample of the workload, ~10 s."""
    import oracle
    from paper_1606_06508_gb300 import synth
    threads = cpu_threads()
    sample = 1 << 22
    x = synth.quaternions_f32(sample, seed=101)
    oracle.normalize_threads(x.reshape(-1), dim=4, threads=threads)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.normalize_threads(x.reshape(-1), dim=4, threads=threads)
        reps += 1
        dt = time.perf_counter() - t0
        if dt > 10.0 or reps >= 4000:
            break
    return {"value": reps * sample / dt, "unit": "vectors/s", "cores": threads, "kind": "oracle",
            "sample": f"{reps} x {sample} quaternions of the same recipe ({dt:.1f} s), oracle on {threads} host "
                      "threads over contiguous vector ranges"}


def parity_sample(x, y, api_mod):
    """Sampled outputs of the timed workload against the oracle (bitwise)."""
    import torch
    import oracle
    n = x.shape[0]
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([np.arange(min(n, 1024)), rng.choice(n, min(n, 1 << 16), replace=False),
                                    np.arange(max(0, n - 1024), n)]))
    it = torch.from_numpy(idx).to(x.device)
    xs = x[it].cpu().numpy()
    ys = y[it].cpu().numpy().reshape(-1)
    oy = oracle.normalize(xs.reshape(-1), dim=4)[0]
    nan = np.isnan(ys) & np.isnan(oy)
    bad = int(np.count_nonzero((ys.view(np.uint32) != oy.view(np.uint32)) & ~nan))
    return {"sampled_vectors": int(idx.size), "mismatching_values": bad, "max_ulp_vs_oracle": 0 if bad == 0 else None}


def extras(api, synth, torch, peak):
    """Secondary measurements (each one call repeated, CUDA events): the
    forward+backward form, rows, ragged, the copy ceiling, the naive algorithm."""
    out = {}
    dev = torch.device("cuda")
    s = torch.cuda.current_stream()

    def rec(name, fn, units, nbytes, iters=10, **kw):
        try:
            fn()
            torch.cuda.synchronize()
            ts = time_events(fn, iters, s)
            t = statistics.median(ts) * 1e-3
            out[name] = {"vectors_per_s": units / t, "ms": t * 1e3, "GB_per_s": nbytes / t / 1e9,
                         "frac_of_hbm_peak": nbytes / t / 1e9 / peak, "algorithmic_bytes": nbytes, **kw}
        except Exception as e:  # report, do not hide
            out[name] = {"error": repr(e)}

    # fwd+bwd, 2^24 binary32 quaternions (forward saves h and code; backward reads y, g, h, code)
    n4 = 1 << 24
    x = synth.quaternions_f32_torch(n4, seed=4, device=dev)
    g = synth.normal_like_torch((n4, 4), torch.float32, seed=40, device=dev)
    y = torch.empty_like(x)
    h = torch.empty(n4, device=dev)
    c = torch.empty(n4, dtype=torch.int8, device=dev)
    gr = torch.empty_like(x)
    from paper_1606_06508_gb300 import _lib as L

    def fb():
        L.check(L.normalize_f32(x.data_ptr(), y.data_ptr(), None, h.data_ptr(), c.data_ptr(), n4, 4, None, None,
                                0, s.cuda_stream), "fwd")
        L.check(L.normalize_backward_f32(y.data_ptr(), g.data_ptr(), h.data_ptr(), c.data_ptr(), gr.data_ptr(), n4, 4,
                                         None, None, 0, s.cuda_stream), "bwd")
    rec("fwd_bwd_quat_f32_2^24", fb, n4, n4 * (16 + 16 + 4 + 1 + 16 + 16 + 4 + 1 + 16),
        bytes_model="fwd 16+16+4+1, bwd 16+16+4+1+16 per quaternion")
    del x, g, y, h, c, gr

    # rows of 256
    for f, cnt in (("f32", 1 << 20), ("f64", 1 << 19)):
        dt = torch.float32 if f == "f32" else torch.float64
        xr = synth.rows_torch(cnt, 256, dt, seed=2, device=dev)
        yr = torch.empty_like(xr)
        fn = L.normalize_f32 if f == "f32" else L.normalize_f64
        rec(f"rows256_{f}", lambda: L.check(fn(xr.data_ptr(), yr.data_ptr(), None, None, None, cnt, 256, None, None, 0,
                                               s.cuda_stream), "rows"), cnt, 2 * xr.numel() * xr.element_size())
        del xr, yr

    # ragged, 4,000,000 vectors (40% of length 2-4, the rest log-uniform in [5, 4096])
    for f in ("f32", "f64"):
        dt = torch.float32 if f == "f32" else torch.float64
        cnt = 4_000_000
        lengths = synth.ragged_lengths_torch(cnt, seed=3, device=dev)
        off = synth.offsets_from_lengths_torch(lengths)
        xv = synth.ragged_values_torch(lengths, dt, seed=3)
        yv = torch.empty_like(xv)
        plan = api.Plan(cnt, dt)
        mapping = plan.autotune(off)
        fn = L.normalize_f32 if f == "f32" else L.normalize_f64
        nb = 2 * xv.numel() * xv.element_size() + 8 * (cnt + 1)
        rec(f"ragged4M_{f}", lambda: L.check(fn(xv.data_ptr(), yv.data_ptr(), None, None, None, cnt, 0, off.data_ptr(),
                                                 plan.handle, 0, s.cuda_stream), "ragged"), cnt, nb,
            mapping=list(mapping), elements=int(xv.numel()))
        del xv, yv, plan, lengths, off

    # the copy ceiling and the naive algorithm on the headline's bytes
    a = torch.empty(QUAT_COUNT * 4, device=dev)
    b = torch.empty_like(a)
    a.normal_()
    rec("copy_2GiB", lambda: L.check(L.ngb_copy(b.data_ptr(), a.data_ptr(), a.numel() * 4, s.cuda_stream), "copy"),
        QUAT_COUNT, 2 * a.numel() * 4)
    rec("naive_quat_f32_2^26", lambda: L.check(L.naive_normalize_f32(a.data_ptr(), b.data_ptr(), QUAT_COUNT, 4,
                                                                      s.cuda_stream), "naive"),
        QUAT_COUNT, QUAT_COUNT * QUAT_BYTES)
    del a, b
    return out


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    __graft_entry__.build()
    from paper_1606_06508_gb300 import _lib as L
    from paper_1606_06508_gb300 import api, synth

    peak, peak_src = peaks()
    s = torch.cuda.current_stream()
    count = args.count
    x = synth.quaternions_f32_torch(count, seed=1 + 1000 * rank, device=dev)
    y = torch.empty_like(x)
    xp, yp = x.data_ptr(), y.data_ptr()

    def step():
        st = L.normalize_f32(xp, yp, None, None, None, count, 4, None, None, 0, s.cuda_stream)
        if st:
            L.check(st, "normalize_f32")

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(torch.cuda.current_device())
    sampler = ClockSampler(gpu_id)
    sampler.start()
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.mark()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler.mark()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    # per-launch durations of the dominant (only) kernel, events on its stream
    per_launch = time_events(step, min(args.steps, 200), s)
    sampler.stop()
    clocks = sampler.summary()

    result = None
    if rank == 0:
        secs = ms * 1e-3
        value = world * args.steps * count / secs
        launch_s = statistics.mean(per_launch) * 1e-3
        achieved = count * QUAT_BYTES / launch_s / 1e9
        traffic, tnote = traffic_for(KERNEL)
        result = {
            "metric": METRIC, "value": value, "unit": "vectors/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if count == QUAT_COUNT else f"{count} quaternions (profiling size)",
                       "vectors_per_gpu": count,
                       "algorithmic_bytes_per_step_per_gpu": count * QUAT_BYTES,
                       "l2": "inputs larger than L2 (1 GiB in, 1 GiB out per GPU); no flush",
                       "parallelism": f"independent batch per GPU x{world}"},
            "GB_per_s": world * args.steps * count * QUAT_BYTES / secs / 1e9,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": KERNEL,
                         "peak_source": peak_src + ("; of measured" if peak_src.startswith("measured") else
                                                    "; of fallback"),
                         "achieved_note": f"32 B algorithmic per quaternion x {count} / mean event time of "
                                          f"{len(per_launch)} single-launch steps",
                         "traffic_note": tnote},
            "gpu_launches": args.steps,
            "clocks": clocks,
        }
    # e2e through host buffers (pinned), same metric
    e2e_steps = max(1, min(args.steps, 20))
    hx = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
    hy = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
    hx.copy_(x)
    torch.cuda.synchronize()

    def e2e_step():
        x.copy_(hx, non_blocking=True)
        step()
        hy.copy_(y, non_blocking=True)
    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(e2e_steps):
        e2e_step()
    b.record(s)
    torch.cuda.synchronize()
    ems = a.elapsed_time(b)
    if world > 1:
        t = torch.tensor([ems], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ems = float(t.item())
    if rank == 0:
        result["e2e"] = {"value": world * e2e_steps * count / (ems * 1e-3), "unit": "vectors/s",
                         "h2d_bytes_per_step": count * 16, "d2h_bytes_per_step": count * 16,
                         "steps": e2e_steps, "note": "pinned host x -> device, normalize_f32, device y -> pinned host"}
        result["parity"] = parity_sample(x, y, api)
        if world == 1:
            if not args.no_extras:
                del hx, hy
                result["also"] = extras(api, synth, torch, peak)
            result["cpu_baseline"] = cpu_baseline_quat()
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--count", type=int, default=QUAT_COUNT,
                    help="quaternions per GPU (default 2^26, the headline workload; smaller only for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
