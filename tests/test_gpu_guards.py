"""Guard-padded launches, the stand-in for a memory checker: every input and
output of one C-ABI call sits between two 512-byte guard zones of a known
byte pattern (tests/guarded.py); after the call the guards must be intact and
every output bit-identical to the oracle.  Tiny configurations: counts 1 to
257, every dimension class of the dense dispatch, bases on and off 16-byte
alignment, ragged batches with empty, length-1, thread-, warp- and
block-sized vectors, forward and backward."""
import numpy as np
import pytest

import guard_cases as gc
from gpu_util import cuda_device
from paper_1606_06508_gb300 import synth

pytestmark = pytest.mark.gpu

DIM_COUNTS = [(1, (1, 2, 257)), (2, (1, 3, 257)), (3, (1, 33, 257)), (4, (1, 2, 31, 257)), (5, (1, 3, 33)),
              (16, (1, 33)), (17, (1, 3)), (33, (2, 9)), (132, (1, 3)), (256, (1, 2, 9)), (257, (1, 3)),
              (1024, (1, 3)), (1025, (1, 2)), (5000, (1, 2)), (16385, (1, 2))]


@pytest.fixture(scope="module")
def env():
    import torch
    dev = cuda_device()
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_06508_gb300 import _lib
    stream = torch.cuda.current_stream().cuda_stream
    return _lib.lib(), stream, torch.cuda.synchronize, dev


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("dim,counts", DIM_COUNTS, ids=[str(d) for d, _ in DIM_COUNTS])
def test_dense_guards_and_parity(env, f, shift, dim, counts):
    lib, stream, sync, dev = env
    for count in counts:
        x = gc.dense_inputs(f, count, dim, seed=dim * 1000 + count)
        fwd = gc.forward_case(lib, stream, sync, dev, f, x, count, dim, shift)
        gc.backward_case(lib, stream, sync, dev, f, fwd, count, dim, shift, seed=count)


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("shift", [0, 1])
def test_ragged_guards_and_parity(env, f, shift):
    from paper_1606_06508_gb300 import api
    lib, stream, sync, dev = env
    for count in gc.RAGGED_COUNTS:
        lengths = gc.ragged_lengths_with_edges(count, seed=count)
        off = synth.offsets_from_lengths(lengths)
        x = synth.ragged_values(lengths, gc.NP[f], seed=count)
        plan = api.Plan(count, gc.TD[f])
        fwd = gc.forward_case(lib, stream, sync, dev, f, x, count, 0, shift, offsets=off, plan=plan.handle)
        gc.backward_case(lib, stream, sync, dev, f, fwd, count, 0, shift, seed=count, offsets=off,
                         plan=plan.handle)
        plan.close()
