"""Benchmark of batched accurate normalization (arXiv 1606.06508) on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload NAME] [--count C] [--no-extras]

Default workload (the headline): one step = one library call on 2^26
binary32 quaternions (1 GiB in, 1 GiB out) normalized with the scaling
algorithm (Algorithm 7).  Inputs are resident in HBM when the timed region
starts and larger than L2, so no flush is needed between steps.  Rank 0 prints
one JSON line with the whole-job throughput (vectors/s), the roofline of the
dominant kernel (algorithmic bytes per launch over its event-timed duration,
against the measured HBM copy bandwidth), the oracle timed on the host cores
on a bounded sample (cpu_baseline), an end-to-end figure through pinned host
buffers (e2e), the SM clocks sampled during the timed region, a bitwise parity
check of sampled outputs against the oracle, and (N = 1, unless --no-extras)
short secondary measurements of the other workloads.

--workload selects another workload of the method for the same JSON line
(per-workload evidence and profiling): fwdbwd_quat, rows_f32, rows_f64,
ragged_f32, ragged_f64, fwdbwd_ragged_f64, vec3_f64, quat_f64.

With N > 1 (torchrun) the ranks share one global batch, each normalizing its
contiguous shard (paper_1606_06508_gb300/shard.py; ragged shards balanced by
element count): strong scaling with no data exchange, the timing the max over
ranks.  --scaling weak gives every rank its own full-size batch instead.

--impl reference times the oracle (plain single-threaded C, run on all host
cores over contiguous vector ranges) on bounded samples of the same workload.
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
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")
L2_BYTES = 126 * 1024 * 1024


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


def quat_bulk_requested() -> bool:
    """The library's opt-in bulk-copy path for binary32 quaternions (read by
    the library once, at its first dense binary32 quaternion call)."""
    return os.environ.get("NGB_QUAT_BULK") == "1"


def traffic_for(workload: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel sources (else None).  The
    summary is of the default kernels: none under the opt-in bulk path."""
    if workload == "quat" and quat_bulk_requested():
        return None, None
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        e = d.get(workload)
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

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
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


def time_events(fn, iters, stream, between=None):
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(iters)]
    for a, b in evs:
        if between:
            between()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


# ---------------------------------------------------------------------------- host samples (oracle side)
def host_sample(name: str, n: int):
    """A bounded host sample of a workload's recipe: (x, dim, offsets, units)."""
    from paper_1606_06508_gb300 import synth
    if name in ("quat", "fwdbwd_quat"):
        x = synth.quaternions_f32(n, seed=101)
        return x.reshape(-1), 4, None, n
    if name in ("rows_f32", "rows_f64"):
        dt = np.float32 if name.endswith("f32") else np.float64
        rows = max(1, n // 256)
        return synth.rows(rows, 256, dt, seed=102).reshape(-1), 256, None, rows
    if name == "quat_f64":
        x = synth.quaternions_f64(n, seed=105)
        return x.reshape(-1), 4, None, n
    if name == "vec3_f64":
        x = synth.vectors3_f64(n, seed=103)
        return x.reshape(-1), 3, None, x.shape[0]
    dt = np.float64 if "f64" in name else np.float32
    kind, nmax = ("loguniform", 1024) if name == "fwdbwd_ragged_f64" else ("mixture", 4096)
    cnt = max(1, n // 300)
    lengths = synth.ragged_lengths(cnt, seed=104, kind=kind, nmax=nmax)
    return synth.ragged_values(lengths, dt, seed=104), 0, synth.offsets_from_lengths(lengths), cnt


def cpu_baseline(name: str, seconds: float = 10.0, single_seconds: float = 3.0):
    """The oracle as it stands, on all host cores over contiguous vector ranges,
    repeated on a bounded sample of the workload for about `seconds`; then the
    same on one thread for about `single_seconds`.  Vectors/s and GB/s (input
    and output values once, plus offsets) for both."""
    import oracle
    oracle.build()
    threads = cpu_threads()
    x, dim, off, units = host_sample(name, 1 << 21)
    nbytes = 2 * x.nbytes + (off.nbytes if off is not None else 0)

    def timed(nthreads, budget):
        oracle.normalize_threads(x, dim, off, threads=nthreads)
        reps, t0 = 0, time.perf_counter()
        while True:
            oracle.normalize_threads(x, dim, off, threads=nthreads)
            reps += 1
            dt = time.perf_counter() - t0
            if dt > budget or reps >= 100000:
                return reps, dt

    reps, dt = timed(threads, seconds)
    reps1, dt1 = timed(1, single_seconds)
    return {"value": reps * units / dt, "unit": "vectors/s", "cores": threads, "kind": "oracle",
            "GB_per_s": reps * nbytes / dt / 1e9,
            "sample": f"{reps} x {units} vectors of the same recipe ({dt:.1f} s, forward), oracle on {threads} "
                      "host threads over contiguous vector ranges",
            "single_thread": {"value": reps1 * units / dt1, "unit": "vectors/s", "cores": 1,
                              "GB_per_s": reps1 * nbytes / dt1 / 1e9,
                              "sample": f"{reps1} x {units} vectors ({dt1:.1f} s), oracle on one thread"}}


# ---------------------------------------------------------------------------- parity of the timed outputs
def _bits_mismatch(a, b):
    ui = np.uint32 if a.dtype == np.float32 else np.uint64
    a, b = a.reshape(-1), b.reshape(-1)
    nan = np.isnan(a) & np.isnan(b)
    return int(np.count_nonzero((a.view(ui) != b.view(ui)) & ~nan))


def parity_full(x, y, dim, off=None, grad=None, g=None):
    """Every output value of the last timed step against the oracle on the same
    inputs (the oracle on all host cores over contiguous vector ranges), after
    the timed region: y, and the gradient of a forward + backward step."""
    import oracle
    threads = cpu_threads()
    t0 = time.perf_counter()
    xh = x.cpu().numpy().reshape(-1)
    offh = off.cpu().numpy() if off is not None else None
    oy, _, oh, oc = oracle.normalize_threads(xh, dim, offh, threads=threads)
    del xh
    bad = _bits_mismatch(y.cpu().numpy(), oy)
    values = int(y.numel())
    if grad is not None:
        og = oracle.backward_threads(oy, g.cpu().numpy().reshape(-1), oh, oc, dim=dim, offsets=offh,
                                     threads=threads)
        bad += _bits_mismatch(grad.cpu().numpy(), og)
        values += int(grad.numel())
    count = oh.size
    return {"vectors": int(count), "values_compared": values, "mismatching_values": bad,
            "max_ulp_vs_oracle": 0 if bad == 0 else None,
            "compared": "every output value of the last timed step (y" + (", grad" if grad is not None else "") +
                        "), bit for bit",
            "oracle_threads": threads, "seconds": time.perf_counter() - t0}


# ---------------------------------------------------------------------------- error vs the exact result
FMT_NAMES = {"f32": "binary32, u = 2^-24", "f64": "binary64, u = 2^-53"}


def _exact_errors(vectors, fmt):
    """Errors (oracle/exact.py, exact rationals and a 256-bit square root) of
    computed (x^, r^) pairs, with the paper's bounds per length: ||x^ - x/r||
    against (3.001 + n/2) u (Lemmas 1, 2, 4; the rounding count of the order
    CR(n) in place of n for n >= 5), |r^ - r| beyond the alpha/2 the lemmas
    allow for a subnormal norm, against (1 + n/2) r u, |sin phi|
    against 1.001 u (Lemma 1, n = 2, 3), and the largest per-component error
    in ulps (no bound in the paper; information).  Zero and non-finite inputs
    are skipped."""
    from oracle import exact
    out = {"direction": {"max_u": 0.0, "max_over_bound": 0.0, "n_at_max": None},
           "norm": {"max_u": 0.0, "max_over_bound": 0.0, "n_at_max": None},
           "sin_phi": {"max_u": 0.0, "bound_u": float(exact.SIN_BOUND_U), "applies_to": "n = 2, 3 (Lemma 1)"},
           "component_ulp_max": 0.0, "vectors_checked": 0, "all_within_bounds": True, "failing_vectors": 0}
    for x, y, r in vectors:
        if not np.all(np.isfinite(x)) or not np.any(x != 0):
            continue
        n = x.size
        e = exact.errors(x, y, r, fmt)
        ok = exact.check(x, y, r, fmt, quaternion=(n == 4)).ok
        out["vectors_checked"] += 1
        if not ok:
            out["all_within_bounds"] = False
            out["failing_vectors"] += 1
        db = float(exact.direction_bound(n, fmt.u))
        d = out["direction"]
        if e["direction_u"] / db > d["max_over_bound"]:
            d["max_over_bound"], d["n_at_max"], d["bound_u_at_max"] = e["direction_u"] / db, n, db
        d["max_u"] = max(d["max_u"], e["direction_u"])
        if e["norm_u"] is not None:
            nb = float(exact.norm_bound(n, fmt.u))
            m = out["norm"]
            if e["norm_u"] / nb > m["max_over_bound"]:
                m["max_over_bound"], m["n_at_max"], m["bound_u_at_max"] = e["norm_u"] / nb, n, nb
            m["max_u"] = max(m["max_u"], e["norm_u"])
        if n in (2, 3):
            out["sin_phi"]["max_u"] = max(out["sin_phi"]["max_u"], e["sin_u"])
        out["component_ulp_max"] = max(out["component_ulp_max"], e["ulp"])
    return out


def accuracy_report(x, y, dim, off=None, k=2000, k_long=200, seed=7, edges=True):
    """Error against the exact result on a seeded sample of the timed output:
    k vectors of n <= 4, k_long longer ones.  The norms come from one more
    library call on the sampled vectors (the timed step writes no norms); its
    y must equal the timed y bit for bit.  With `edges`, the 64 binary64 edge
    vectors of the 3-vector workload are normalized by the library and checked
    the same way."""
    import torch
    from oracle import exact
    from paper_1606_06508_gb300 import api, synth
    t0 = time.perf_counter()
    rng = np.random.default_rng(seed)
    fmt = exact.F32 if x.dtype == torch.float32 else exact.F64
    if off is None:
        count = x.numel() // dim
        kk = min(count, k if dim <= 4 else k_long)
        idx = np.sort(rng.choice(count, kk, replace=False))
        it = torch.from_numpy(idx).to(x.device)
        xs = x.reshape(count, dim)[it].contiguous()
        ys = y.reshape(count, dim)[it]
        ys2, rs = api.normalize(xs, return_norm=True)
        lens = np.full(kk, dim)
        sub = synth.offsets_from_lengths(lens)
    else:
        offh = off.cpu().numpy()
        count = offh.size - 1
        n = np.diff(offh)
        short, long_ = np.flatnonzero(n <= 4), np.flatnonzero(n > 4)
        idx = np.sort(np.concatenate([rng.choice(short, min(k, short.size), replace=False),
                                      rng.choice(long_, min(k_long, long_.size), replace=False)]))
        lens = n[idx]
        sub = synth.offsets_from_lengths(lens)
        gather = np.concatenate([np.arange(offh[i], offh[i + 1]) for i in idx]).astype(np.int64)
        gt = torch.from_numpy(gather).to(x.device)
        xs, ys = x[gt].contiguous(), y[gt]
        ys2, rs = api.normalize(xs, torch.from_numpy(sub).to(x.device), return_norm=True)
    torch.cuda.synchronize()
    consistent = _bits_mismatch(ys2.cpu().numpy(), ys.cpu().numpy()) == 0
    xh, yh, rh = xs.cpu().numpy().reshape(-1), ys.cpu().numpy().reshape(-1), rs.cpu().numpy()
    vecs = [(xh[sub[i]:sub[i + 1]], yh[sub[i]:sub[i + 1]], rh[i]) for i in range(lens.size)]
    rep = {"format": FMT_NAMES["f32" if fmt is exact.F32 else "f64"],
           "sample": f"{lens.size} vectors of the timed output (seed {seed}; n <= 4: up to {k}, longer: up to "
                     f"{k_long})",
           "norms_from_a_second_call_consistent": bool(consistent),
           **_exact_errors(vecs, fmt)}
    if edges:
        e = synth.edge_vectors_d3_f64()
        ye, re_ = api.normalize(torch.from_numpy(e).to(x.device), return_norm=True)
        torch.cuda.synchronize()
        ye, re_ = ye.cpu().numpy(), re_.cpu().numpy()
        rep["edge_vectors_d3_f64"] = _exact_errors([(e[i], ye[i], re_[i]) for i in range(e.shape[0])], exact.F64)
    rep["seconds"] = time.perf_counter() - t0
    return rep


# ---------------------------------------------------------------------------- workloads
class Work:
    """One workload: a step (device-resident inputs), its units and algorithmic
    bytes, the dominant kernel, host buffers for the end-to-end figure, and
    for binary64 the algorithmic FP64 operations per step."""

    def __init__(self, **kw):
        self.flush = False
        self.dp_ops = None
        self.__dict__.update(kw)
        ptrs = {k: t.data_ptr() for k, t in self.arrays.items()}
        self.step = lambda: self.launch(ptrs)


DP_OPS_MODEL = ("binary64 operations of the paper's sequence done on the FP64 pipe: 3 per element (square, "
                "sum, output product) + 3 per vector (square root, reciprocal, norm product); backward 5 per "
                "element (product, sum, product, difference, product); exact power-of-two scalings not counted")


def fp64_rate(torch, L):
    """Measured binary64 multiply + add rate of this GPU (FP64 operations per
    second): ngb_fp64_probe, one wave of 8 blocks per SM, median of 5 timed launches."""
    import ctypes
    blocks = 8 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    ops = ctypes.c_int64(0)
    s = torch.cuda.current_stream()

    def fn():
        L.check(L.ngb_fp64_probe(out.data_ptr(), blocks, 1024, ctypes.byref(ops), s.cuda_stream), "fp64 probe")
    fn()
    torch.cuda.synchronize()
    t = statistics.median(time_events(fn, 5, s)) * 1e-3
    return ops.value / t


def dp_roofline(w, ms_per_step, rate):
    """FP64-pipe bound of a binary64 step next to its byte bound."""
    if w.dp_ops is None or not rate:
        return None
    bound_ms = w.dp_ops / rate * 1e3
    return {"dp_ops_per_step": w.dp_ops, "fp64_ops_per_s": rate, "bound_ms": bound_ms,
            "measured_ms": ms_per_step, "frac": bound_ms / ms_per_step, "ops_model": DP_OPS_MODEL,
            "peak_source": "measured live: ngb_fp64_probe (dmul + dadd chains)"}


def _dense_shard(t, part):
    """Rows [a, b) of t for part = (world, rank) (shard.dense_range); t itself
    without a part."""
    if part is None:
        return t
    from paper_1606_06508_gb300 import shard
    a, b = shard.dense_range(t.shape[0], *part)
    return t[a:b].contiguous()


def _ragged_shard(off, tensors, part):
    """The vectors [a, b) of a ragged batch for part = (world, rank), balanced
    by element count (shard.ragged_range): their offsets rebased to 0 and the
    slices of the packed arrays."""
    if part is None:
        return off, tensors
    from paper_1606_06508_gb300 import shard
    offh = off.cpu().numpy()
    a, b = shard.ragged_range(offh, *part)
    s0, s1 = int(offh[a]), int(offh[b])
    return (off[a:b + 1] - s0).contiguous(), [t[s0:s1].contiguous() for t in tensors]


def build_work(name, count, rank, torch, L, api, synth, mapping=None, part=None):
    """The workload `name`: its arrays (device tensors), `launch(p)` running
    one step of library calls on the pointers p[name] (so that the same step
    runs on device buffers or, for the end-to-end figure, on pinned host
    buffers), which arrays are the step's inputs and results, its units and
    algorithmic bytes, and the post-timing checks.  With part = (world, rank)
    every rank draws the same global batch and keeps its shard of it (strong
    scaling, no exchange between ranks); otherwise each rank draws its own
    full-size batch (weak scaling)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    s = torch.cuda.current_stream()
    seed = 0 if part is not None else 1000 * rank

    if name == "quat":
        x = _dense_shard(synth.quaternions_f32_torch(count, seed=1 + seed, device=dev), part)
        y = torch.empty_like(x)
        nq = x.shape[0]

        def launch(p):
            st = L.normalize_f32(p["x"], p["y"], None, None, None, nq, 4, None, None, 0, s.cuda_stream)
            if st:
                L.check(st, "normalize_f32")
        return Work(desc=("2^26 binary32 quaternions (float4 AoS), forward: Algorithm 7, 50/50 "
                          "wide-exponent/N(0,1) components") if count == QUAT_COUNT
                    else f"{count} binary32 quaternions, forward (profiling size)",
                    units=nq, global_units=count, bytes=32 * nq, dtype="f32",
                    kernel="k_quat_bulk (NGB_QUAT_BULK=1)" if quat_bulk_requested() else "k_small_vec16<float,4>",
                    launches=1,
                    arrays={"x": x, "y": y}, inputs=["x"], results=["y"], launch=launch,
                    parity=lambda: parity_full(x, y, 4), accuracy=lambda: accuracy_report(x, y, 4),
                    bytes_model="16 B read + 16 B written per quaternion")

    if name == "fwdbwd_quat":
        n_glob = count if count != QUAT_COUNT else 1 << 24
        x = _dense_shard(synth.quaternions_f32_torch(n_glob, seed=4 + seed, device=dev), part)
        g = _dense_shard(synth.normal_like_torch((n_glob, 4), torch.float32, seed=40 + seed, device=dev), part)
        n = x.shape[0]
        y, gr = torch.empty_like(x), torch.empty_like(x)
        h = torch.empty(n, device=dev)
        c = torch.empty(n, dtype=torch.int8, device=dev)

        def launch(p):
            L.check(L.normalize_f32(p["x"], p["y"], None, p["h"], p["c"], n, 4, None, None, 0, s.cuda_stream), "fwd")
            L.check(L.normalize_backward_f32(p["y"], p["g"], p["h"], p["c"], p["gr"], n, 4, None, None, 0,
                                             s.cuda_stream), "bwd")
        return Work(desc=f"{n} binary32 quaternions, forward (saving h and code) + backward",
                    units=n, global_units=n_glob, bytes=90 * n, dtype="f32",
                    kernel="k_small_vec16<float,4> + k_small_bwd<float,4>",
                    launches=2, arrays={"x": x, "g": g, "y": y, "h": h, "c": c, "gr": gr}, inputs=["x", "g"],
                    results=["gr"], launch=launch,
                    parity=lambda: parity_full(x, y, 4, grad=gr, g=g), accuracy=lambda: accuracy_report(x, y, 4),
                    bytes_model="fwd 16+16+4+1, bwd 16+16+4+1+16 per quaternion")

    if name in ("rows_f32", "rows_f64"):
        dt = torch.float32 if name.endswith("f32") else torch.float64
        rows_glob = count if count != QUAT_COUNT else (1 << 20 if dt == torch.float32 else 1 << 19)
        x = _dense_shard(synth.rows_torch(rows_glob, 256, dt, seed=2 + seed, device=dev), part)
        rows = x.shape[0]
        y = torch.empty_like(x)
        fn = L.normalize_f32 if dt == torch.float32 else L.normalize_f64

        def launch(p):
            L.check(fn(p["x"], p["y"], None, None, None, rows, 256, None, None, 0, s.cuda_stream), "rows")
        return Work(desc=f"{rows} rows of 256 {name[-3:]}, forward, N(0,1) x 2^s per row",
                    units=rows, global_units=rows_glob, bytes=2 * x.numel() * x.element_size(), dtype=name[-3:],
                    kernel=('k_rows_half<4>' if dt == torch.float32 else 'k_rows_stream_batch<double,4>'), launches=1,
                    arrays={"x": x, "y": y}, inputs=["x"], results=["y"], launch=launch,
                    parity=lambda: parity_full(x, y, 256), accuracy=lambda: accuracy_report(x, y, 256),
                    bytes_model="2 x 256 x s per row",
                    dp_ops=(3 * rows * 256 + 3 * rows) if dt == torch.float64 else None)

    if name in ("ragged_f32", "ragged_f64", "fwdbwd_ragged_f64"):
        dt = torch.float64 if "f64" in name else torch.float32
        fb = name.startswith("fwdbwd")
        cnt_glob = count if count != QUAT_COUNT else (500_000 if fb else 4_000_000)
        kind, nmax = ("loguniform", 1024) if fb else ("mixture", 4096)
        lengths = synth.ragged_lengths_torch(cnt_glob, seed=3 + seed, kind=kind, nmax=nmax, device=dev)
        off = synth.offsets_from_lengths_torch(lengths)
        x = synth.ragged_values_torch(lengths, dt, seed=3 + seed)
        g = synth.normal_like_torch(x.shape, dt, seed=41 + seed, device=dev) if fb else None
        off, parts = _ragged_shard(off, [x, g] if fb else [x], part)
        x, g = (parts[0], parts[1]) if fb else (parts[0], None)
        cnt = off.numel() - 1
        y = torch.empty_like(x)
        plan = api.Plan(cnt, dt)
        if mapping:  # a fixed mapping (profiling): no autotuning launches before the timed ones
            plan.set_mapping(*mapping)
            mapping = plan.mapping
        else:
            mapping = plan.autotune(off)
        fn = L.normalize_f32 if dt == torch.float32 else L.normalize_f64
        s_bytes = x.element_size()
        if not fb:
            def launch(p):
                L.check(fn(p["x"], p["y"], None, None, None, cnt, 0, p["off"], plan.handle, 0, s.cuda_stream),
                        "ragged")
            return Work(desc=f"{cnt} ragged {name[-3:]} vectors (40% of length 2-4, else log-uniform [5,4096]), "
                             f"int64 offsets, forward, one persistent launch after the classifier",
                        units=cnt, global_units=cnt_glob, bytes=2 * x.numel() * s_bytes + 8 * (cnt + 1),
                        dtype=name[-3:],
                        kernel="k_classify + k_ragged (persistent)", launches=2,
                        arrays={"x": x, "off": off, "y": y}, inputs=["x", "off"], results=["y"], launch=launch,
                        parity=lambda: parity_full(x, y, 0, off=off), accuracy=lambda: accuracy_report(x, y, 0, off=off),
                        mapping=list(mapping), plan=plan,
                        bytes_model="2 n s per vector + 8 B offsets",
                        dp_ops=(3 * x.numel() + 3 * cnt) if dt == torch.float64 else None)
        gr = torch.empty_like(x)
        h = torch.empty(cnt, dtype=dt, device=dev)
        c = torch.empty(cnt, dtype=torch.int8, device=dev)

        def launch(p):
            L.check(fn(p["x"], p["y"], None, p["h"], p["c"], cnt, 0, p["off"], plan.handle, 0, s.cuda_stream), "fwd")
            L.check(L.normalize_backward_f64(p["y"], p["g"], p["h"], p["c"], p["gr"], cnt, 0, p["off"], plan.handle, 0,
                                             s.cuda_stream), "bwd")
        return Work(desc=f"{cnt} ragged binary64 vectors, lengths log-uniform [2,1024], forward + backward",
                    units=cnt, global_units=cnt_glob, bytes=5 * x.numel() * s_bytes + 2 * 9 * cnt + 2 * 8 * (cnt + 1),
                    dtype="f64",
                    kernel="k_classify + k_ragged; k_classify + k_ragged_bwd_{blocks,warps,threads}", launches=6,
                    arrays={"x": x, "g": g, "off": off, "y": y, "h": h, "c": c, "gr": gr},
                    inputs=["x", "g", "off"], results=["gr"], launch=launch,
                    parity=lambda: parity_full(x, y, 0, off=off, grad=gr, g=g),
                    accuracy=lambda: accuracy_report(x, y, 0, off=off),
                    mapping=list(mapping), plan=plan,
                    bytes_model="fwd 2ns + 9 + 8, bwd 3ns + 9 + 8 per vector",
                    dp_ops=8 * x.numel() + 3 * cnt)

    if name == "quat_f64":
        n_glob = count if count != QUAT_COUNT else 1 << 25
        x = _dense_shard(synth.quaternions_f64_torch(n_glob, seed=5 + seed, device=dev), part)
        n = x.shape[0]
        y = torch.empty_like(x)

        def launch(p):
            L.check(L.normalize_f64(p["x"], p["y"], None, None, None, n, 4, None, None, 0, s.cuda_stream), "quat_f64")
        return Work(desc=f"{n} binary64 quaternions (components sign x U[1,2) x 2^e, e in [-30,30]), forward",
                    units=n, global_units=n_glob, bytes=64 * n, dtype="f64", kernel="k_small_direct<double,4>",
                    launches=1,
                    arrays={"x": x, "y": y}, inputs=["x"], results=["y"], launch=launch,
                    parity=lambda: parity_full(x, y, 4), accuracy=lambda: accuracy_report(x, y, 4),
                    bytes_model="32 B read + 32 B written per quaternion", dp_ops=15 * n)

    if name == "vec3_f64":
        xh = synth.vectors3_f64(65536, seed=0 + seed)
        x = _dense_shard(torch.from_numpy(xh).to(dev), part)
        y = torch.empty_like(x)
        cnt = x.shape[0]

        def launch(p):
            L.check(L.normalize_f64(p["x"], p["y"], None, None, None, cnt, 3, None, None, 0, s.cuda_stream), "vec3")
        return Work(desc="65,536 x 3 binary64 vectors (e in [-30,30]) + 64 edge vectors, forward",
                    units=cnt, global_units=xh.shape[0], bytes=48 * cnt, dtype="f64",
                    kernel="k_small_direct<double,3>", launches=1,
                    arrays={"x": x, "y": y}, inputs=["x"], results=["y"], launch=launch,
                    parity=lambda: parity_full(x, y, 3), accuracy=lambda: accuracy_report(x, y, 3, k=4000),
                    flush=True, bytes_model="24 B read + 24 B written per vector", dp_ops=12 * cnt)
    raise ValueError(f"unknown workload {name}")


def full_size_desc(name):
    """The workload description of the full-size line, shared by both arms."""
    return {
        "quat": "2^26 binary32 quaternions (float4 AoS), forward: Algorithm 7, 50/50 wide-exponent/N(0,1) components",
        "fwdbwd_quat": f"{1 << 24} binary32 quaternions, forward (saving h and code) + backward",
        "rows_f32": f"{1 << 20} rows of 256 f32, forward, N(0,1) x 2^s per row",
        "rows_f64": f"{1 << 19} rows of 256 f64, forward, N(0,1) x 2^s per row",
        "ragged_f32": "4000000 ragged f32 vectors (40% of length 2-4, else log-uniform [5,4096]), int64 offsets, "
                      "forward, one persistent launch after the classifier",
        "ragged_f64": "4000000 ragged f64 vectors (40% of length 2-4, else log-uniform [5,4096]), int64 offsets, "
                      "forward, one persistent launch after the classifier",
        "fwdbwd_ragged_f64": "500000 ragged binary64 vectors, lengths log-uniform [2,1024], forward + backward",
        "vec3_f64": "65,536 x 3 binary64 vectors (e in [-30,30]) + 64 edge vectors, forward",
        "quat_f64": f"{1 << 25} binary64 quaternions (components sign x U[1,2) x 2^e, e in [-30,30]), forward",
    }[name]


WORKLOAD_NAMES = ["quat", "fwdbwd_quat", "rows_f32", "rows_f64", "ragged_f32", "ragged_f64", "fwdbwd_ragged_f64",
                  "vec3_f64", "quat_f64"]


def paper_tables(torch, L, synth, s):
    """GPU analogues of the paper's Tables 3 and 4 (Appendix A): on 2^24
    three-component vectors with N(0,1) components, the time of the quotient
    Algorithms 1 and 2 over the time of the scaling algorithm (Table 3), and
    the time of the scaling algorithm over the naive sequence (Table 4);
    CUDA events, median of 10 launches each."""
    out = {}
    n = 1 << 24
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        x = synth.normal_like_torch((n, 3), dt, seed=77, device="cuda")
        y = torch.empty_like(x)
        r = torch.empty(n, dtype=dt, device="cuda")
        xp, yp, rp = x.data_ptr(), y.data_ptr(), r.data_ptr()
        norm = L.normalize_f32 if name == "f32" else L.normalize_f64
        quot = L.quotient_normalize3_f32 if name == "f32" else L.quotient_normalize3_f64
        naive = L.naive_normalize_f32 if name == "f32" else L.naive_normalize_f64
        fns = {
            "scaling": lambda: L.check(norm(xp, yp, rp, None, None, n, 3, None, None, 0, s.cuda_stream), "scaling"),
            "scaling_no_norm": lambda: L.check(norm(xp, yp, None, None, None, n, 3, None, None, 0, s.cuda_stream),
                                               "scaling"),
            "quotient_alg1": lambda: L.check(quot(xp, yp, rp, n, 1, s.cuda_stream), "alg1"),
            "quotient_alg2": lambda: L.check(quot(xp, yp, rp, n, 2, s.cuda_stream), "alg2"),
            "naive": lambda: L.check(naive(xp, yp, n, 3, s.cuda_stream), "naive"),
        }
        ms = {}
        for k, fn in fns.items():
            fn()
            torch.cuda.synchronize()
            ms[k] = statistics.median(time_events(fn, 10, s))
        out[f"paper_tables_vec3_{name}"] = {
            "vectors": n, "ms": ms,
            "table3_time_quotient_over_scaling": {"alg1": ms["quotient_alg1"] / ms["scaling"],
                                                  "alg2": ms["quotient_alg2"] / ms["scaling"]},
            "table4_time_scaling_over_naive": ms["scaling_no_norm"] / ms["naive"],
            "note": "Table 3: scaling and quotient algorithms return y and r; Table 4: both return y only"}
        del x, y, r
        torch.cuda.empty_cache()
    return out


def extras(torch, L, api, synth, peak, rate):
    """Secondary measurements on this GPU (each step repeated 10 times,
    CUDA events): the other workloads, the copy ceiling, the naive algorithm."""
    out = {}
    s = torch.cuda.current_stream()
    for name in WORKLOAD_NAMES[1:]:
        try:
            w = build_work(name, QUAT_COUNT, 0, torch, L, api, synth)
            w.step()
            torch.cuda.synchronize()
            flush = None
            if w.flush:
                fb = torch.empty(2 * L2_BYTES // 4, device="cuda")
                flush = lambda: fb.fill_(1.0)  # noqa: E731
            t = statistics.median(time_events(w.step, 10, s, between=flush)) * 1e-3
            out[name] = {"vectors_per_s": w.units / t, "ms": t * 1e3, "GB_per_s": w.bytes / t / 1e9,
                         "frac_of_hbm_peak": w.bytes / t / 1e9 / peak, "algorithmic_bytes": w.bytes,
                         "kernel": w.kernel, **({"mapping": w.mapping} if hasattr(w, "mapping") else {})}
            dp = dp_roofline(w, t * 1e3, rate)
            if dp:
                out[name]["dp_roofline"] = dp
            del w
        except Exception as e:  # report, do not hide
            out[name] = {"error": repr(e)}
        torch.cuda.empty_cache()
    out.update(paper_tables(torch, L, synth, s))
    a = torch.empty(QUAT_COUNT * 4, device="cuda")
    b = torch.empty_like(a)
    a.normal_()
    for nm, fn, units, nb in (
            ("copy_2GiB", lambda: L.check(L.ngb_copy(b.data_ptr(), a.data_ptr(), a.numel() * 4, s.cuda_stream), "c"),
             QUAT_COUNT, 2 * a.numel() * 4),
            ("naive_quat_f32_2^26", lambda: L.check(L.naive_normalize_f32(a.data_ptr(), b.data_ptr(), QUAT_COUNT, 4,
                                                                           s.cuda_stream), "n"),
             QUAT_COUNT, 32 * QUAT_COUNT)):
        fn()
        t = statistics.median(time_events(fn, 10, s)) * 1e-3
        out[nm] = {"vectors_per_s": units / t, "ms": t * 1e3, "GB_per_s": nb / t / 1e9,
                   "frac_of_hbm_peak": nb / t / 1e9 / peak, "algorithmic_bytes": nb}
    return out


# ---------------------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = cpu_threads()
    x, dim, off, units = host_sample(args.workload, 1 << 17)
    for _ in range(args.warmup):
        oracle.normalize_threads(x, dim, off, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.normalize_threads(x, dim, off, threads=threads)
    dt = time.perf_counter() - t0
    v = args.steps * units / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "vectors/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None,
        "dtype": "f64" if args.workload.endswith("f64") else "f32", "data": "synthetic",
        "config": {"workload": full_size_desc(args.workload), "workload_name": args.workload,
                   "reference_step": f"{units} vectors of the same recipe (bounded sample)"},
        "cpu_baseline": {"value": v, "unit": "vectors/s", "cores": threads, "kind": "oracle",
                         "sample": f"{units} vectors per step, oracle on {threads} host threads over contiguous ranges"},
        "e2e": {"value": v, "unit": "vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- our arm
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
    strong = args.scaling == "strong"
    w = build_work(args.workload, args.count, rank, torch, L, api, synth, mapping=args.mapping,
                   part=(world, rank) if strong and world > 1 else None)
    # units all ranks process per step: the global batch (strong), or world full batches (weak)
    job_units = w.global_units if strong else world * w.units
    flush = None
    if w.flush:
        flush_buf = torch.empty(2 * L2_BYTES // 4, device=dev)
        flush = lambda: flush_buf.fill_(1.0)  # noqa: E731

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(torch.cuda.current_device())
    sampler = ClockSampler(gpu_id)
    sampler.start()
    warm = max(args.warmup, 3)
    for _ in range(warm):
        w.step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.mark()
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            w.step()
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    else:  # L2 flushed between steps, outside the timed intervals
        ms = sum(time_events(w.step, args.steps, s, between=flush))
    if world > 1:
        torch.distributed.barrier()
    sampler.mark()
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    # per-step durations, events on the launching stream
    per_step = time_events(w.step, min(args.steps, 200), s, between=flush)
    sampler.stop()
    clocks = sampler.summary()

    result = None
    if rank == 0:
        secs = ms * 1e-3
        step_s = statistics.mean(per_step) * 1e-3
        achieved = w.bytes / step_s / 1e9
        traffic, tnote = traffic_for(args.workload)
        result = {
            "metric": METRIC, "value": args.steps * job_units / secs, "unit": "vectors/s", "n_gpus": world,
            "steps": args.steps, "warmup": warm, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": args.scaling, "vs_baseline": None, "dtype": w.dtype, "data": "synthetic",
            "config": {"workload": full_size_desc(args.workload) if args.count == QUAT_COUNT else w.desc,
                       "workload_name": args.workload,
                       "vectors_per_gpu": w.units, "algorithmic_bytes_per_step_per_gpu": w.bytes,
                       "bytes_model": w.bytes_model,
                       "l2": ("L2 flushed between steps (256 MB write), outside the timed intervals" if w.flush else
                              "inputs larger than L2 (126 MB); no flush"),
                       "parallelism": (f"one global batch of {w.global_units} vectors sharded over {world} GPU(s) by "
                                       "contiguous vector ranges (ragged: balanced by element count), no exchange"
                                       if strong else f"independent full-size batch per GPU x{world}"),
                       **({"mapping": w.mapping} if hasattr(w, "mapping") else {})},
            "GB_per_s": world * args.steps * w.bytes / secs / 1e9,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": w.kernel,
                         "peak_source": peak_src + ("; of measured" if peak_src.startswith("measured") else
                                                    "; of fallback"),
                         "achieved_note": f"algorithmic bytes per step / mean event time of {len(per_step)} steps "
                                          f"({w.launches} kernel launch(es) per step)",
                         "traffic_note": tnote},
            "gpu_launches": args.steps * w.launches,
            "clocks": clocks,
        }
        need_rate = w.dp_ops is not None or (world == 1 and not args.no_extras and args.workload == "quat")
        rate = fp64_rate(torch, L) if need_rate else None
        if rate:
            result["fp64_ops_per_s"] = rate
        dp = dp_roofline(w, ms / args.steps, rate)
        if dp:
            result["dp_roofline"] = dp
    if args.kernels_only:
        if rank == 0:
            result["kernels_only"] = True
            print(json.dumps(result), flush=True)
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0
    # e2e through the library's public calls with the step's inputs and results
    # in pinned host memory.  Main figure: the calls are given the host
    # pointers, and the kernels read the inputs and write the results over the
    # host link (NVLink-C2C) themselves -- the host-to-device and device-to-host
    # transfers happen inside every timed step, with no staging copy.  Beside
    # it: the same step staged by copy engines (inputs copied to the device,
    # the device call, results copied back).
    e2e_steps = max(1, min(args.steps, 20))
    host = {k: torch.empty(w.arrays[k].shape, dtype=w.arrays[k].dtype, pin_memory=True)
            for k in w.inputs + w.results}
    for k in w.inputs:
        host[k].copy_(w.arrays[k])
    zptrs = {k: t.data_ptr() for k, t in w.arrays.items()}
    zptrs.update({k: t.data_ptr() for k, t in host.items()})
    torch.cuda.synchronize()

    def zero_copy_step():
        w.launch(zptrs)

    def staged_step():
        for k in w.inputs:
            w.arrays[k].copy_(host[k], non_blocking=True)
        w.step()
        for k in w.results:
            host[k].copy_(w.arrays[k], non_blocking=True)

    def time_e2e(fn):
        fn()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(e2e_steps):
            fn()
        b.record(s)
        torch.cuda.synchronize()
        t_ms = a.elapsed_time(b)
        if world > 1:
            t = torch.tensor([t_ms], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            t_ms = float(t.item())
        return t_ms

    zms = time_e2e(zero_copy_step)
    zero_copy_results = {k: host[k].clone() for k in w.results}
    sms = time_e2e(staged_step)  # leaves the device step's results in host[k]
    same = all(_bits_mismatch(zero_copy_results[k].numpy(), host[k].numpy()) == 0 for k in w.results)
    if rank == 0:
        h2d = sum(host[k].numel() * host[k].element_size() for k in w.inputs)
        d2h = sum(host[k].numel() * host[k].element_size() for k in w.results)
        result["e2e"] = {"value": e2e_steps * job_units / (zms * 1e-3), "unit": "vectors/s",
                         "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                         "ms_per_step": zms / e2e_steps,
                         "link_GB_per_s": (h2d + d2h) * e2e_steps / (zms * 1e-3) / 1e9,
                         "note": "inputs and results in pinned host memory; the library calls get the host pointers "
                                 "and their kernels read the inputs and write the results over the host link "
                                 "(zero-copy), inside every timed step",
                         "results_equal_device_path": bool(same),
                         "staged": {"value": e2e_steps * job_units / (sms * 1e-3), "unit": "vectors/s",
                                    "ms_per_step": sms / e2e_steps,
                                    "note": "copy engines: pinned host inputs -> device, the device call(s), device "
                                            "results -> pinned host, one after the other"}}
        result["parity"] = w.parity()
        result["accuracy"] = w.accuracy()
        if world == 1:
            if not args.no_extras and args.workload == "quat":
                del host, zero_copy_results
                w = None
                torch.cuda.empty_cache()
                result["also"] = extras(torch, L, api, synth, peak, rate)
            result["cpu_baseline"] = cpu_baseline(args.workload)
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
    ap.add_argument("--workload", choices=WORKLOAD_NAMES, default="quat")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--scaling", choices=["strong", "weak"], default="strong",
                    help="with N > 1: strong = every rank takes its shard of one global batch (shard.py ranges, no "
                         "exchange); weak = every rank normalizes its own full-size batch")
    ap.add_argument("--kernels-only", action="store_true",
                    help="profiling: time the steps and print the line without the end-to-end figure, the checks "
                         "and the CPU baseline")
    ap.add_argument("--mapping", type=lambda v: [int(t) for t in v.split(",")], default=None,
                    help="ragged workloads: thread_max,warp_max,block_threads,grid_blocks instead of autotuning "
                         "(profiling)")
    ap.add_argument("--count", type=int, default=QUAT_COUNT,
                    help="units per GPU; the default selects each workload's full size (2^26 quaternions for the "
                         "headline); smaller values only for profiling")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
