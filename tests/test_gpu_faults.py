"""Failure handling without any GPU fault: host-side injected errors (misaligned
pointers, non-finite parameters) return error codes and leave the problem
usable; a non-finite training step is skipped; and a device-side wait that runs
out (a barrier nothing completes) gives up, reports NBM_ERR_DEVICE_TIMEOUT and
leaves the context usable.  Nothing here traps, faults or hangs the GPU.
"""
import ctypes as C
import time

import numpy as np
import pytest
import torch

from tests import inputs

pytestmark = pytest.mark.gpu


def _prob():
    import paper_2210_14907_gb300 as nbm
    d = nbm.ProblemDesc(geometry=nbm.GEOM_SPHERE, n_hidden=2, width=64)
    return nbm, nbm.Problem(d)


def test_bounded_device_wait_gives_up_and_the_device_stays_usable():
    nbm, prob = _prob()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    rc = prob.lib.nbm_selftest_bounded_wait(200_000_000, stream)  # ~0.1 s at 2 GHz
    wall = time.perf_counter() - t0
    assert rc == 6, nbm._lib.nbm_last_error()
    assert wall < 5.0
    th = torch.from_numpy(inputs.glorot_params(64, 2, seed=3)).cuda()
    loss, g = prob.loss_grad(th, n=4096)
    assert np.isfinite(loss) and torch.isfinite(g).all()
    rc = prob.lib.nbm_selftest_bounded_wait(10, stream)
    assert rc == 1


def test_misaligned_pointers_are_rejected():
    nbm, prob = _prob()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    th = torch.from_numpy(inputs.glorot_params(64, 2, seed=4)).cuda()
    raw = torch.zeros(4 * prob.P + 64, dtype=torch.uint8, device="cuda")
    odd = C.c_void_p(raw.data_ptr() + 2)
    grad = torch.zeros(prob.P, device="cuda")
    loss = C.c_double()
    L = prob.lib
    assert L.nbm_loss_grad(prob.handle, odd, None, 1024, 1, 1, C.c_void_p(grad.data_ptr()),
                           C.byref(loss), stream) == 1
    assert L.nbm_loss_grad(prob.handle, C.c_void_p(th.data_ptr()), None, 1024, 1, 1, odd,
                           C.byref(loss), stream) == 1
    assert L.nbm_residual(prob.handle, C.c_void_p(th.data_ptr()), odd, 16, 1, 1, None,
                          C.byref(loss), stream) == 1
    assert "aligned" in nbm._lib.nbm_last_error().decode()
    ok, _ = prob.loss_grad(th, n=1024)  # still usable
    assert np.isfinite(ok)


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_non_finite_parameters_report_nonfinite(bad):
    nbm, prob = _prob()
    th = torch.from_numpy(inputs.glorot_params(64, 2, seed=5)).cuda()
    th[7] = bad
    with pytest.raises(nbm.NBMError) as e:
        prob.loss_grad(th, n=1024)
    assert e.value.code == 4


def test_a_non_finite_training_step_is_skipped():
    nbm, prob = _prob()
    th = torch.from_numpy(inputs.glorot_params(64, 2, seed=6)).cuda()
    th[3] = float("nan")
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    hist = torch.zeros(3, device="cuda")
    before = th.clone()
    s = prob.train_steps(th, m, v, 0, 3, 2048, seed=1, loss_hist=hist)
    torch.cuda.synchronize()
    assert s == 3
    assert torch.isnan(hist).all()
    assert torch.equal(m, torch.zeros_like(m)) and torch.equal(v, torch.zeros_like(v))
    assert torch.equal(torch.nan_to_num(th), torch.nan_to_num(before))  # no update applied
    th[3] = 0.1
    hist2 = torch.zeros(5, device="cuda")
    prob.train_steps(th, m, v, s, 5, 2048, seed=1, loss_hist=hist2)
    assert torch.isfinite(hist2).all() and torch.isfinite(th).all()
