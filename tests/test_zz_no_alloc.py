"""nbm_loss_grad_static, the entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc while they run: hosts whose
own pool or arena owns all device memory (plugins, inference servers),
real-time or embedded hosts that forbid allocation after start-up, and code
that must not synchronize the device as cudaMalloc and cudaFree may.  Its
scratch is one static device array inside libnbm.  Its results are checked
against the FP64 oracle and against the allocating nbm_loss_grad.

This file runs last (pytest collects it last), so a failure here leaves every
other test already run.  It passes both alone in a fresh process and after the
rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from tests import inputs

pytestmark = pytest.mark.gpu


def _static_entry(lib):
    fn = lib.nbm_loss_grad_static
    P = ctypes.c_void_p
    fn.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int64, P,
                   ctypes.POINTER(ctypes.c_double), P]
    fn.restype = ctypes.c_int
    return fn


@pytest.mark.parametrize("prec, loss_tol, grad_tol", [(0, 1e-5, 1e-4), (1, 2e-3, 5e-3)],
                         ids=["fp32", "bf16"])
def test_static_scratch_matches_allocating_entry_point_twice(prec, loss_tol, grad_tol):
    import paper_2210_14907_gb300 as nbm
    d = nbm.ProblemDesc(geometry=nbm.GEOM_FLOWER, n_hidden=3, width=128, precision=prec,
                        mu_minus=1.0, mu_plus=100.0, h=2.0 / 128)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=O.GEOM_FLOWER, n_hidden=3, width=128, mu_minus=1.0,
                       mu_plus=100.0, h=2.0 / 128)
    fn = _static_entry(prob.lib)
    stream = torch.cuda.current_stream()
    for call in range(2):
        p32 = inputs.mixed_points(3000, 1000, seed=40 + call).astype(np.float32)
        pts = torch.from_numpy(p32).cuda()
        th_np = inputs.glorot_params(128, 3, seed=call, bias_scale=0.1)
        th = torch.from_numpy(th_np).cuda()
        loss_o, g_o = O.loss_grad(o, th_np.astype(np.float64), p32.astype(np.float64))
        loss_ref, g_ref = prob.loss_grad(th, pts)
        g = torch.full((prob.P,), float("nan"), device="cuda")
        loss = ctypes.c_double(0.0)
        rc = fn(prob.handle, ctypes.c_void_p(th.data_ptr()), ctypes.c_void_p(pts.data_ptr()),
                pts.shape[0], 1, 1, ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss),
                ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, prob.lib.nbm_last_error()
        torch.cuda.synchronize()
        g = g.cpu().numpy().astype(np.float64)
        g_ref = g_ref.cpu().numpy().astype(np.float64)
        # against the FP64 oracle, within the path's tolerances
        assert abs(loss.value - loss_o) / loss_o <= loss_tol
        assert np.linalg.norm(g - g_o) / np.linalg.norm(g_o) <= grad_tol
        # and against the allocating entry point on the same inputs
        assert abs(loss.value - loss_ref) / loss_ref <= loss_tol
        assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= grad_tol


def test_static_scratch_rejects_oversized_batch():
    import paper_2210_14907_gb300 as nbm
    prob = nbm.Problem(nbm.config("C1"))
    fn = _static_entry(prob.lib)
    th = torch.zeros(prob.P, device="cuda")
    g = torch.zeros(prob.P, device="cuda")
    rc = fn(prob.handle, ctypes.c_void_p(th.data_ptr()), None, 16385, 1, 1,
            ctypes.c_void_p(g.data_ptr()), None, None)
    assert rc == 1
    assert b"static-scratch limit" in prob.lib.nbm_last_error()


def test_static_entry_allocates_no_device_memory():
    """Repeated calls on a problem whose workspace was never allocated leave
    the device's free memory unchanged; the allocating entry point on another
    fresh problem does change it (the check sees a workspace allocation)."""
    import paper_2210_14907_gb300 as nbm
    d = nbm.config("C2")
    prob = nbm.Problem(d)  # fresh: nothing of its own allocated yet
    fn = _static_entry(prob.lib)
    n = 8192
    pts = torch.from_numpy(inputs.mixed_points(n - 2000, 2000, seed=5).astype(np.float32)).cuda()
    th = torch.from_numpy(inputs.glorot_params(128, 3, seed=5, bias_scale=0.1)).cuda()
    g = torch.empty(prob.P, device="cuda")
    stream = torch.cuda.current_stream()
    args = (prob.handle, ctypes.c_void_p(th.data_ptr()), ctypes.c_void_p(pts.data_ptr()), n, 1, 1,
            ctypes.c_void_p(g.data_ptr()), None, ctypes.c_void_p(stream.cuda_stream))
    assert fn(*args) == 0, prob.lib.nbm_last_error()  # warm: the library is loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert fn(*args) == 0, prob.lib.nbm_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # control: the allocating entry point reserves its workspace on first use
    other = nbm.Problem(d)
    lg = other.lib.nbm_loss_grad  # argument types as the package declares them
    assert lg(other.handle, th.data_ptr(), pts.data_ptr(), n, 1, 1, g.data_ptr(), None,
              stream.cuda_stream) == 0, other.lib.nbm_last_error()
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 < free1
