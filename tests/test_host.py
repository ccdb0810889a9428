"""Host-side checks that need no GPU: the C ABI library builds, loads and
exports every entry point of include/normgb.h; argument errors are reported
before any CUDA work; the product code never touches the oracle; the header
is plain C; the multi-rank sharding logic partitions a batch (gloo,
world_size 2, each rank running the oracle on its shard)."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "normgb.h")
PKG = os.path.join(ROOT, "paper_1606_06508_gb300")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_06508_gb300 import build
    build.build()
    from paper_1606_06508_gb300 import _lib
    return _lib


def test_header_is_plain_c():
    for lang, std in (("c", "c99"), ("c++", "c++11")):
        r = subprocess.run(["gcc", "-fsyntax-only", "-Wall", "-Werror", "-x", lang, f"-std={std}", HEADER],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_symbol(lib):
    names = header_functions()
    assert "normalize_f32" in names and "normalize_backward_f64" in names and "ngb_plan_create" in names
    raw = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing
    assert set(names) <= set(lib.PROTOTYPES), set(names) - set(lib.PROTOTYPES)


def test_argument_errors_before_any_cuda_work(lib):
    L = lib
    f32 = L.normalize_f32
    assert f32(None, None, None, None, None, -1, 4, None, None, 0, None) == L.NGB_ERR_INVALID_ARG
    assert f32(1, 1, None, None, None, 4, -2, None, None, 0, None) == L.NGB_ERR_INVALID_ARG
    assert f32(1, 1, None, None, None, 4, (1 << 20) + 1, None, None, 0, None) == L.NGB_ERR_UNSUPPORTED
    assert f32(1, 1, None, None, None, 4, 4, None, None, 0x80, None) == L.NGB_ERR_INVALID_ARG
    assert f32(1, 1, None, None, None, 4, 4, 8, None, 0, None) == L.NGB_ERR_INVALID_ARG  # offsets with dim > 0
    assert f32(1, 1, None, None, None, 4, 0, None, None, 0, None) == L.NGB_ERR_INVALID_ARG  # ragged, no offsets
    assert f32(1, 1, None, None, None, 4, 0, 8, None, 0, None) == L.NGB_ERR_NO_PLAN
    assert "plan" in L.last_error()
    assert f32(None, None, None, None, None, 0, 4, None, None, 0, None) == L.NGB_OK  # count 0: no-op
    assert f32(None, 1, None, None, None, 3, 4, None, None, 0, None) == L.NGB_ERR_INVALID_ARG  # x NULL
    b = L.normalize_backward_f64
    assert b(1, 1, 1, None, 1, 3, 4, None, None, 0, None) == L.NGB_ERR_INVALID_ARG  # saved_code NULL
    assert L.ngb_plan_create(10, 2, 0)[0] == L.NGB_ERR_UNSUPPORTED
    assert L.ngb_plan_create(-1, 4, 0)[0] == L.NGB_ERR_INVALID_ARG
    assert L.ngb_plan_create(1 << 31, 4, 0)[0] == L.NGB_ERR_UNSUPPORTED
    assert L.naive_normalize_f32(1, 1, 5, 7, None) == L.NGB_ERR_INVALID_ARG
    assert L.ngb_copy(1, 1, -5, None) == L.NGB_ERR_INVALID_ARG
    assert L.normalize_to_rotation_f32(None, None, None, -1, None) == L.NGB_ERR_INVALID_ARG


def test_no_gpu_reports_cuda_error_not_crash(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, p = lib.ngb_plan_create(10, 4, 0)
    assert st == lib.NGB_ERR_CUDA and p is None and lib.last_error()


def test_missing_library_fails_loudly(tmp_path):
    code = ("import paper_1606_06508_gb300._lib as L; L.LIB_PATH = '/nonexistent/libnormgb.so'; "
            "import sys\ntry:\n    L.lib()\nexcept ImportError as e:\n    print('IMPORTERROR', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert "IMPORTERROR" in r.stdout, r.stdout + r.stderr


def test_package_import_is_lazy():
    code = ("import sys, paper_1606_06508_gb300, paper_1606_06508_gb300.synth; "
            "print('LOADED' if 'paper_1606_06508_gb300._lib' in sys.modules and "
            "sys.modules['paper_1606_06508_gb300._lib']._lib is not None else 'LAZY')")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert "LAZY" in r.stdout, r.stdout + r.stderr


def test_product_never_touches_the_oracle():
    """The library, its binding and the input generators share nothing with
    oracle/, and the oracle includes nothing of the library."""
    for dirpath, _, files in os.walk(PKG):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"\b(import|from)\s+oracle\b|\boracle\.\w|#include[^\n]*oracle", text), \
                    f"{fn} uses the oracle"
    for fn in ("normalize_oracle.c", "oracle_impl.h", "__init__.py"):
        text = open(os.path.join(ROOT, "oracle", fn)).read()
        assert "csrc" not in text and "normgb" not in text and "paper_1606_06508_gb300" not in text, fn


def test_synth_holds_no_method_arithmetic():
    text = open(os.path.join(PKG, "synth.py")).read()
    for word in ("sqrt", "tau_", "sigma", "rcp", "normalize("):
        assert word not in text, word


# ----------------------------------------------------------------------------- sharding
def test_shard_ranges_partition():
    from paper_1606_06508_gb300 import shard, synth
    for count in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            rs = [shard.dense_range(count, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == count
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
    lengths = synth.ragged_lengths(20000, seed=3)
    off = synth.offsets_from_lengths(lengths)
    for world in (2, 4, 8):
        rs = [shard.ragged_range(off, world, r) for r in range(world)]
        assert rs[0][0] == 0 and rs[-1][1] == len(lengths)
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
        elems = [off[b] - off[a] for a, b in rs]
        assert max(elems) - min(elems) <= 2 * 4096 + off[-1] // 100


def test_shard_range_matches_its_definition(lib):
    """ngb_shard_range against the definition written out: dense, the floor of
    count * rank / world; ragged, the first vector whose start is at least
    offsets[0] + floor(total * rank / world) (offsets not starting at 0, empty
    vectors included); argument errors."""
    import numpy as np
    L = lib
    rng = np.random.default_rng(5)
    for count in (0, 1, 2, 7, 1000, 2 ** 40):
        for world in (1, 2, 3, 8, 13):
            for rank in range(world):
                st, a, b = L.ngb_shard_range(None, count, world, rank)
                assert st == L.NGB_OK and (a, b) == (count * rank // world, count * (rank + 1) // world)
    for trial in range(30):
        count = int(rng.integers(0, 300))
        lengths = rng.integers(0, 50, size=count)
        lengths[rng.random(count) < 0.2] = 0
        start = int(rng.integers(0, 100))
        off = (start + np.concatenate([[0], np.cumsum(lengths)])).astype(np.int64)
        total = int(off[-1] - off[0])
        for world in (1, 2, 5, 8):
            bounds = []
            for rank in range(world):
                st, a, b = L.ngb_shard_range(off.ctypes.data, count, world, rank)
                assert st == L.NGB_OK
                def cut(r):
                    if r <= 0:
                        return 0
                    if r >= world:
                        return count
                    target = int(off[0]) + total * r // world
                    return next((i for i in range(count) if off[i] >= target), count)
                assert (a, b) == (cut(rank), cut(rank + 1)), (trial, world, rank)
                bounds.append((a, b))
            assert bounds[0][0] == 0 and bounds[-1][1] == count
            assert all(bounds[i][1] == bounds[i + 1][0] for i in range(world - 1))
            if count:
                assert all(abs(int(off[b] - off[a]) - total / world) <= int(lengths.max()) for a, b in bounds)
    assert L.ngb_shard_range(None, 5, 0, 0)[0] == L.NGB_ERR_INVALID_ARG
    assert L.ngb_shard_range(None, 5, 2, 2)[0] == L.NGB_ERR_INVALID_ARG
    assert L.ngb_shard_range(None, -1, 2, 0)[0] == L.NGB_ERR_INVALID_ARG


def _gloo_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1606_06508_gb300 import shard, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lengths = synth.ragged_lengths(3000, seed=3, nmax=600)
    off = synth.offsets_from_lengths(lengths)
    x = synth.ragged_values(lengths, np.float64, seed=3)
    a, b = shard.ragged_range(off, world, rank)
    sub_off = off[a:b + 1] - off[a]
    y = oracle.normalize(x[off[a]:off[b]], dim=0, offsets=sub_off)[0]
    parts = [None] * world
    dist.all_gather_object(parts, (a, b, y))
    if rank == 0:
        full = np.concatenate([p[2] for p in sorted(parts, key=lambda t: t[0])])
        ref = oracle.normalize(x, dim=0, offsets=off)[0]
        # each shard's element count is within one vector's length of an even split
        elems = [int(off[b_] - off[a_]) for a_, b_, _ in parts]
        balanced = all(abs(e - int(off[-1]) / world) <= int(lengths.max()) for e in elems)
        q.put(bool(np.array_equal(full, ref)) and parts[0][1] == parts[1][0] and balanced)
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_shard_and_gather():
    import torch.multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True


def test_bench_shards_partition_one_global_batch():
    """bench.py's strong-scaling shards (the ranges of shard.py): the ranks'
    slices concatenate to the global batch, each ragged shard's offsets start
    at 0 and describe its slice, and element counts stay within one vector's
    length of an even split."""
    import torch
    sys.path.insert(0, ROOT)
    import bench
    from paper_1606_06508_gb300 import synth
    x = torch.arange(1001 * 4, dtype=torch.float32).reshape(1001, 4)
    lengths = synth.ragged_lengths(5000, seed=3)
    off = torch.from_numpy(synth.offsets_from_lengths(lengths))
    v = torch.arange(int(off[-1]), dtype=torch.float64)
    g = -v
    for world in (1, 2, 3, 8):
        parts = [bench._dense_shard(x, (world, r)) for r in range(world)]
        assert torch.equal(torch.cat(parts), x)
        vs, gs = [], []
        for r in range(world):
            o, (vr, gr) = bench._ragged_shard(off, [v, g], (world, r))
            assert int(o[0]) == 0 and int(o[-1]) == vr.numel() == gr.numel()
            assert abs(vr.numel() - int(off[-1]) / world) <= int(lengths.max())
            vs.append(vr)
            gs.append(gr)
        assert torch.equal(torch.cat(vs), v) and torch.equal(torch.cat(gs), g)
    assert bench._dense_shard(x, None) is x
