"""gs_loss_l1_noalloc -- the L1 loss entry point for callers that may not
allocate device memory (their memory belongs to a host framework's pool, or
they run where allocation is not allowed).  It must give the same loss and
gradient as the workspace-based gs_loss_l1, call after call, although every
call reuses the same static scratch array inside the library.

This file is collected last on purpose: it checks a call that shares state
across calls, so it runs after every other test (and also alone).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_00219_gb300 import build
    build.build()
    from paper_2605_00219_gb300 import gsstep
    return gsstep


def _reference(gsstep, image, target, w, h):
    """Loss and gradient from the workspace-based entry point gs_loss_l1."""
    plan = gsstep.Plan([1], [(w, h, 0)])
    ws = torch.empty(plan.workspace_bytes(), dtype=torch.uint8, device="cuda")
    gsstep.gs_workspace_init(plan, ws)
    dl = torch.empty_like(image)
    gsstep.gs_loss_l1(plan, ws, image, target, dl)
    return dl, gsstep.gs_read_stats(plan, ws).loss


def test_noalloc_matches_workspace_l1_twice(gs):
    gsstep = gs
    w, h = 333, 217                      # not a multiple of the block size
    rng = np.random.default_rng(0)
    loss_dev = torch.zeros(1, dtype=torch.float32, device="cuda")
    for call in range(2):                # two calls in a row share the scratch
        image = torch.from_numpy(rng.uniform(0, 1, size=(h * w, 3)).astype(np.float32)).cuda()
        target = torch.from_numpy(rng.uniform(0, 1, size=(h * w, 3)).astype(np.float32)).cuda()
        target[:100] = image[:100]       # some exact ties (sign 0)
        dl_ref, loss_ref = _reference(gsstep, image, target, w, h)
        dl = torch.full_like(image, 7.0)
        gsstep.gs_loss_l1_noalloc(image, target, dl, loss_dev)
        torch.cuda.synchronize()
        assert torch.equal(dl, dl_ref), call
        assert float(loss_dev.item()) == pytest.approx(loss_ref, rel=1e-6, abs=0), call
        assert float(loss_dev.item()) == pytest.approx(
            float((image.double() - target.double()).abs().mean()), rel=1e-5)


def test_noalloc_rejects_sizes_beyond_its_maximum(gs):
    gsstep = gs
    lib = gsstep.lib()
    big = gsstep.L1_NOALLOC_MAX_VALUES + 1
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    rc = lib.gs_loss_l1_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), big, None)
    assert rc == 1  # GS_ERR_INVALID_ARG, nothing launched
    rc = lib.gs_loss_l1_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 0, None)
    assert rc == 1


def test_noalloc_inside_a_captured_graph(gs):
    """After a warm-up call (which looks up the scratch address), the entry
    point can be captured in a CUDA graph; replays give the eager results."""
    gsstep = gs
    w, h = 257, 129
    rng = np.random.default_rng(1)
    image = torch.from_numpy(rng.uniform(0, 1, size=(h * w, 3)).astype(np.float32)).cuda()
    target = torch.from_numpy(rng.uniform(0, 1, size=(h * w, 3)).astype(np.float32)).cuda()
    dl_ref, loss_ref = _reference(gsstep, image, target, w, h)
    loss_dev = torch.zeros(1, dtype=torch.float32, device="cuda")
    dl = torch.zeros_like(image)
    gsstep.gs_loss_l1_noalloc(image, target, dl, loss_dev)          # warm-up, eager
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        gsstep.gs_loss_l1_noalloc(image, target, dl, loss_dev, stream=s)
    for _ in range(2):
        dl.fill_(7.0)
        loss_dev.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(dl, dl_ref)
        assert float(loss_dev.item()) == pytest.approx(loss_ref, rel=1e-6, abs=0)


def test_workspace_l1_on_unaligned_and_ragged_buffers(gs):
    """gs_loss_l1 reads four values at a time when the three buffers are
    16-byte aligned and one at a time otherwise; both give the closed form
    on a value count that is not a multiple of 4."""
    gsstep = gs
    w, h = 101, 37
    n = 3 * w * h
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 1, size=n).astype(np.float32)
    tgt = rng.uniform(0, 1, size=n).astype(np.float32)
    tgt[:50] = img[:50]
    ref_dl = np.sign(img - tgt).astype(np.float32) / np.float32(n)
    ref_loss = float(np.abs(img.astype(np.float64) - tgt.astype(np.float64)).mean())
    plan = gsstep.Plan([1], [(w, h, 0)])
    ws = torch.empty(plan.workspace_bytes(), dtype=torch.uint8, device="cuda")
    for shift in (0, 1):                       # 0: aligned, 1: 4-byte offset
        bi = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
        bt = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
        bd = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
        image, target, dl = bi[shift:shift + n], bt[shift:shift + n], bd[shift:shift + n]
        image.copy_(torch.from_numpy(img))
        target.copy_(torch.from_numpy(tgt))
        gsstep.gs_workspace_init(plan, ws)
        gsstep.gs_loss_l1(plan, ws, image, target, dl)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dl.cpu().numpy(), ref_dl)
        assert gsstep.gs_read_stats(plan, ws).loss == pytest.approx(ref_loss, rel=1e-5)
