"""The bounds-checked build (libgsstep_debug.so, compiled with GS_DEBUG).

Indices that the kernels read from the workspace (tile ranges, pair and
emission-slot indices, bucket slots) are checked before they address memory;
a bad one sets GS_STATUS_BOUNDS and the access is skipped.  Each case runs in
a child process that loads the debug library (GS_DEBUG_LIB=1):

- a training step of the tiny workload gives status 0 and the same keys,
  image, gradient records and updated parameters, bit for bit, as the
  normal library;
- with one tile's list range pointing past the intersection capacity (written
  into the workspace on the host after the sort), the debug raster forward and
  backward report GS_STATUS_BOUNDS and treat that list as empty.  This case
  runs only against the debug library, whose entry check of every range keeps
  the access inside the buffers.
"""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

CHILD = r'''
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
from paper_2605_00219_gb300 import gsstep, step, synth
assert gsstep.LIB_PATH.endswith("libgsstep_debug.so"), gsstep.LIB_PATH
mode, out = sys.argv[2], sys.argv[3]
torch.cuda.set_device(0)
scene, _, cams = synth.tiny_workload(0)
tr = step.Trainer([scene], cams, lr=(1e-3,) * 6)
g = torch.Generator(device="cuda").manual_seed(3)
tr.target.copy_(torch.rand(tr.target.shape, device="cuda", generator=g))
if mode == "clean":
    tr.step(step=1)
    torch.cuda.synchronize()
    st = tr.stats()
    K = int(st.k_required)
    np.savez(out, status=st.status, keys=tr.buffer(2, K).cpu().numpy(), image=tr.image.cpu().numpy(),
             grads=gsstep.gs_gradient_records(tr.plan, tr.ws, K).cpu().numpy(), geom=tr.scenes[0].geom.cpu().numpy())
else:
    tr.forward()
    torch.cuda.synchronize()
    tiles, cap = tr.plan.tiles, tr.plan.capacity
    rg = tr.buffer(4, 2 * tiles).view(tiles, 2)
    rg[5, 0] = 0
    rg[5, 1] = cap + 4096
    gsstep.gs_raster_fwd(tr.plan, tr.ws, tr.bg, tr.image)
    tr.dl.copy_(torch.rand(tr.dl.shape, device="cuda", generator=g) - 0.5)
    gsstep.gs_raster_bwd(tr.plan, tr.ws, tr.image, tr.dl)
    torch.cuda.synchronize()
    nl = tr.buffer(5, 128 * 128).cpu().numpy().reshape(128, 128)
    np.savez(out, status=tr.stats().status, nlast_tile5=nl[0:16, 80:96])
'''


@pytest.fixture(scope="module")
def debug_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_00219_gb300 import build
    build.build()
    return build.build(debug=True)


def _child(mode, tmp):
    out = os.path.join(tmp, f"{mode}.npz")
    env = dict(os.environ, GS_DEBUG_LIB="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, mode, out], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


def test_debug_build_equals_normal_build(debug_lib):
    from paper_2605_00219_gb300 import gsstep, step, synth
    assert gsstep.LIB_PATH.endswith("libgsstep.so")
    scene, _, cams = synth.tiny_workload(0)
    tr = step.Trainer([scene], cams, lr=(1e-3,) * 6)
    g = torch.Generator(device="cuda").manual_seed(3)
    tr.target.copy_(torch.rand(tr.target.shape, device="cuda", generator=g))
    tr.step(step=1)
    torch.cuda.synchronize()
    st = tr.stats()
    K = int(st.k_required)
    with tempfile.TemporaryDirectory() as tmp:
        d = _child("clean", tmp)
    assert int(d["status"]) == 0 and st.status == 0
    np.testing.assert_array_equal(d["keys"], tr.buffer(2, K).cpu().numpy())
    np.testing.assert_array_equal(d["image"], tr.image.cpu().numpy())
    np.testing.assert_array_equal(d["grads"], gsstep.gs_gradient_records(tr.plan, tr.ws, K).cpu().numpy())
    np.testing.assert_array_equal(d["geom"], tr.scenes[0].geom.cpu().numpy())


def test_debug_build_reports_a_range_past_the_capacity(debug_lib):
    with tempfile.TemporaryDirectory() as tmp:
        d = _child("corrupt", tmp)
    from paper_2605_00219_gb300 import gsstep
    assert int(d["status"]) & gsstep.STATUS_BOUNDS
    assert not d["nlast_tile5"].any()        # the list was treated as empty
