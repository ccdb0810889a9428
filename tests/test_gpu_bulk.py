"""The opt-in bulk-copy quaternion kernel (csrc/ngb_bulk.cuh, NGB_QUAT_BULK=1):
a child process with the variable set normalizes binary32 quaternion batches
whose sizes fall below one tile, on tile edges and past them (with zeros,
NaN, infinities and subnormals among the components); every output must equal
the oracle's bits, and the path's state word (ngb_quat_bulk_state) must say
that the bulk kernel ran and that no wait gave up.  The variable is read once
per process, hence the child; this process, without it, must not take the
path."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from gpu_util import assert_bits, cuda_device

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COUNTS = [1, 5, 1023, 1024, 1025, 4 * 1024 + 17, 37 * 1024, (1 << 20) + 3]

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1606_06508_gb300 import api, synth
out_dir, counts = sys.argv[2], json.loads(sys.argv[3])
specials = np.array([[0, 0, 0, 0], [np.nan, 1, 2, 3], [np.inf, 0, 0, 0], [1e-45, 0, 0, 0],
                     [3e38, -3e38, 3e38, 1], [0, 0, -0.0, 0]], dtype=np.float32)
for count in counts:
    x = synth.quaternions_f32_torch(count, seed=count, device="cuda")
    k = min(count, specials.shape[0])
    x[:k] = torch.from_numpy(specials[:k]).cuda()
    y, r, h, c = api.normalize(x, return_norm=True, save=True)
    torch.cuda.synchronize()
    np.savez(f"{out_dir}/q{count}.npz", x=x.cpu().numpy(), y=y.cpu().numpy(), r=r.cpu().numpy(),
             h=h.cpu().numpy(), c=c.cpu().numpy())
import ctypes
from paper_1606_06508_gb300 import _lib as L
st = ctypes.c_uint32(0)
assert L.lib().ngb_quat_bulk_state(ctypes.byref(st)) == L.NGB_OK
print(json.dumps({"state": int(st.value)}))
"""


@pytest.fixture(scope="module")
def dev():
    d = cuda_device()
    import __graft_entry__
    __graft_entry__.build()
    return d


def test_bulk_path_is_off_by_default(dev):
    import ctypes
    import torch
    from paper_1606_06508_gb300 import _lib as L
    from paper_1606_06508_gb300 import api, synth
    if os.environ.get("NGB_QUAT_BULK") == "1":
        pytest.skip("NGB_QUAT_BULK=1 in this process")
    x = synth.quaternions_f32_torch(5000, seed=9, device=dev)
    api.normalize(x)
    torch.cuda.synchronize()
    st = ctypes.c_uint32(7)
    L.check(L.lib().ngb_quat_bulk_state(ctypes.byref(st)), "ngb_quat_bulk_state")
    assert st.value == 0


def test_bulk_quaternions_match_oracle(dev, tmp_path):
    env = dict(os.environ, NGB_QUAT_BULK="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path), json.dumps(COUNTS)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    state = json.loads(r.stdout.strip().splitlines()[-1])["state"]
    assert state == 1, state  # the bulk kernel ran; no wait gave up
    for count in COUNTS:
        d = np.load(tmp_path / f"q{count}.npz")
        oy, orr, oh, oc = oracle.normalize(d["x"].reshape(-1), dim=4)
        for name, got, ref in (("y", d["y"], oy), ("norm", d["r"], orr), ("h", d["h"], oh), ("code", d["c"], oc)):
            assert_bits(got.reshape(-1), np.asarray(ref).reshape(-1), f"bulk count={count} {name}")
