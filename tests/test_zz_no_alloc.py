"""cg_l1_loss_static: the L1 loss for callers that cannot allocate device
memory (no workspace; the reduction scratch is a static device array).
Checked through the C ABI against cg_l1_loss on two calls in a row, the
second with different data, so stale scratch from the first call cannot
leak into the second.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_03775_gb300 import cg, scenes

pytestmark = pytest.mark.gpu


def _static_fn(lib):
    fn = lib.cg_l1_loss_static
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def test_static_l1_matches_workspace_l1_twice():
    lib = cg.load()
    fn = _static_fn(lib)
    scene, cams, _ = scenes.config_tiny()
    r = cg.Renderer(cams)
    r.forward(cg.SceneTensors.from_scene(scene))   # a workspace for the reference entry point
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(123)
    for count in (3 * 1957 * 1091, 100_003):
        a = torch.from_numpy(rng.normal(size=count).astype(np.float32)).cuda()
        b = torch.from_numpy(rng.normal(size=count).astype(np.float32)).cuda()
        loss_ref, d_ref = r.l1_loss(a, b)
        d_new = torch.full_like(a, 7.0)
        loss_new = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        st = fn(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), count,
                ctypes.c_void_p(d_new.data_ptr()), ctypes.c_void_p(loss_new.data_ptr()), stream)
        assert st == cg.CG_OK
        torch.cuda.synchronize()
        assert abs(loss_new.item() - loss_ref.item()) <= 1e-12 * max(1.0, abs(loss_ref.item()))
        assert torch.equal(d_new, d_ref)


def test_static_l1_rejects_oversize_and_bad_args():
    fn = _static_fn(cg.load())
    x = torch.zeros(4, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert fn(p, p, (1 << 26) + 1, p, ctypes.c_void_p(loss.data_ptr()), None) == cg.CG_ERR_ARG
    assert fn(p, p, 0, p, ctypes.c_void_p(loss.data_ptr()), None) == cg.CG_ERR_ARG
    assert fn(None, p, 4, p, ctypes.c_void_p(loss.data_ptr()), None) == cg.CG_ERR_ARG
