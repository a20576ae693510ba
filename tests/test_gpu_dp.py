"""Data-parallel training through libnbm (Sec. 3: points distributed over
processors, locally computed gradients aggregated).

- One rank (no exchange) reproduces nbm_train_steps bitwise.
- Shards that partition a batch sum to the whole batch's loss and gradient
  (FP32 reduction order only), and a drawn shard holds exactly the whole
  batch's points at its positions, band points included.
- Two processes on one GPU, exchanging over gloo (host copies, so no kernel
  waits on the other process), train like one process on the whole batch and
  keep bitwise-identical replicas; their first gradient matches the FP64
  oracle's whole-batch gradient.
- nbm_adam_step skips a step whose loss is not finite and refuses bad
  arguments.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import pyoracle as O
from tests import inputs

pytestmark = pytest.mark.gpu


def _nbm():
    import paper_2210_14907_gb300 as nbm
    return nbm


@pytest.mark.parametrize("name, batch", [("C2", 16384), ("C3", 20000)])
def test_single_rank_reproduces_train_steps_bitwise(name, batch):
    nbm = _nbm()
    from paper_2210_14907_gb300.data_parallel import DataParallelTrainer
    d = nbm.config(name)
    prob = nbm.Problem(d)
    p0 = nbm.xavier_init(d, seed=3, device="cuda")
    a = p0.clone()
    ma, va = torch.zeros_like(a), torch.zeros_like(a)
    hist = torch.zeros(3, device="cuda")
    prob.train_steps(a, ma, va, 0, 3, batch, seed=5, loss_hist=hist)
    b = p0.clone()
    mb, vb = torch.zeros_like(b), torch.zeros_like(b)
    tr = DataParallelTrainer(prob, b, mb, vb, batch, seed=5)
    losses = [float(tr.step().item()) for _ in range(3)]
    assert tr.t == 3
    for x, y in ((a, b), (ma, mb), (va, vb)):
        assert torch.equal(x, y)
    assert np.allclose(losses, hist.cpu().numpy(), rtol=1e-7, atol=0)


@pytest.mark.parametrize("name, batch", [("C2", 16384), ("C3", 20000)])
def test_shards_sum_to_the_whole_batch(name, batch):
    nbm = _nbm()
    from paper_2210_14907_gb300.data_parallel import shard_range
    d = nbm.config(name)
    prob = nbm.Problem(d)
    p0 = nbm.xavier_init(d, seed=3, device="cuda")
    lf, gf = prob.loss_grad(p0, n=batch, seed=5, step=4)
    gs = torch.zeros_like(p0)
    ls = 0.0
    for r in range(3):  # uneven shards: batch is not a multiple of 3
        f, n = shard_range(batch, 3, r)
        loss, g = prob.loss_grad_shard(p0, batch, f, n, seed=5, step=4)
        gs += g
        ls += float(loss.item())
    # per-point values do not depend on the partition (the drawn shard below is
    # bitwise the batch's points): loss and gradient differ by the order of the
    # FP32 partial sums only
    assert abs(ls - lf) <= 1e-6 * lf
    assert (torch.linalg.norm(gs - gf) / torch.linalg.norm(gf)).item() <= 1e-5
    # the last shard (the band points of C3 included) holds the whole batch's points
    allp = prob.sample_points(batch, seed=5, step=4)
    f, n = shard_range(batch, 3, 2)
    l_drawn, _ = prob.loss_grad_shard(p0, batch, f, n, seed=5, step=4)
    l_given, _ = prob.loss_grad_shard(p0, batch, f, n, seed=5, step=4,
                                      pts=allp[f:f + n].contiguous())
    assert l_drawn.item() == l_given.item()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir, batch, steps):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2210_14907_gb300 as nbm
        from paper_2210_14907_gb300.data_parallel import DataParallelTrainer, torch_all_reduce
        torch.cuda.set_device(0)
        d = nbm.config("C2")
        prob = nbm.Problem(d)
        p = torch.from_numpy(inputs.glorot_params(128, 3, seed=2, bias_scale=0.1)).cuda()
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        tr = DataParallelTrainer(prob, p, m, v, batch, rank=rank, world=world,
                                 all_reduce=torch_all_reduce(), seed=7)
        # the first step's all-reduced gradient, kept for the oracle check
        loss = tr.step()
        g1 = tr.grad.cpu().numpy().copy()
        losses = [float(loss.item())]
        for _ in range(steps - 1):
            losses.append(float(tr.step().item()))
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), p=p.cpu().numpy(), m=m.cpu().numpy(),
                 v=v.cpu().numpy(), g1=g1, losses=np.array(losses))
    finally:
        dist.destroy_process_group()


def test_two_processes_train_like_one_on_the_whole_batch(tmp_path):
    nbm = _nbm()
    world, batch, steps = 2, 8192, 3
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), batch, steps),
                       nprocs=world, start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    for k in ("p", "m", "v", "g1", "losses"):
        assert np.array_equal(r0[k], r1[k]), k  # replicas identical on both ranks
    # one process, the whole batch
    d = nbm.config("C2")
    prob = nbm.Problem(d)
    th = inputs.glorot_params(128, 3, seed=2, bias_scale=0.1)
    p = torch.from_numpy(th).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    hist = torch.zeros(steps, device="cuda")
    _, g1 = prob.loss_grad(p, n=batch, seed=7, step=1)
    prob.train_steps(p, m, v, 0, steps, batch, seed=7, loss_hist=hist)
    g1 = g1.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(r0["g1"] - g1) / np.linalg.norm(g1) <= 1e-5
    h = hist.cpu().numpy()
    assert abs(r0["losses"][0] - h[0]) <= 1e-6 * h[0]  # the same parameters, FP32 loss history
    assert np.allclose(r0["losses"][1:], h[1:], rtol=1e-5, atol=0)
    pp = p.cpu().numpy()
    # Adam normalises each component (a step of about lr * sign(g) at first), so
    # a component whose gradient is within FP32 reduction order of zero can move
    # the other way; every other component agrees to reduction order
    diff = np.abs(r0["p"] - pp)
    print(f"DP params: max diff {diff.max():.3e}, share > 1e-6: {np.mean(diff > 1e-6):.2e}, "
          f"rel norm {np.linalg.norm(r0['p'] - pp) / np.linalg.norm(pp):.2e}")
    assert np.mean(diff > 1e-6) <= 1e-3
    assert diff.max() <= 2 * steps * 1e-3 + 1e-6
    # the aggregated gradient against the FP64 oracle's whole-batch gradient
    o = O.make_problem(geometry=O.GEOM_SPHERE, n_hidden=3, width=128, mu_minus=1.0,
                       mu_plus=10.0, h=2.0 / 128)
    pts = O.sample_points(o, 7, 1, batch, 0)
    _, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
    assert np.linalg.norm(r0["g1"] - g_ref) / np.linalg.norm(g_ref) <= 5e-3


def test_adam_step_skips_a_non_finite_loss_and_checks_arguments():
    nbm = _nbm()
    prob = nbm.Problem(nbm.config("C1"))
    p = torch.from_numpy(inputs.glorot_params(64, 2, seed=1)).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    g = torch.ones_like(p)
    bad = torch.tensor([float("nan")], dtype=torch.float64, device="cuda")
    before = p.clone()
    assert prob.adam_step(p, m, v, g, 0, loss=bad) == 1
    torch.cuda.synchronize()
    assert torch.equal(p, before) and not m.any() and not v.any()
    ok = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    assert prob.adam_step(p, m, v, g, 1, loss=ok) == 2
    # update 2 with m, v zero so far: m = 0.1, v = 0.001, bias-corrected to 0.1/0.19 and
    # 0.001/0.001999 -> a step of lr * 0.5263 / 0.7073 on every component
    step = (before - p).cpu().numpy()
    c1, c2 = 1 - 0.9 ** 2, 1 - 0.999 ** 2
    expect = 1e-3 * (0.1 / c1) / (np.sqrt(0.001 / c2) + 1e-8)
    assert np.allclose(step, expect, rtol=1e-5)
    with pytest.raises(nbm.NBMError) as e:
        prob.adam_step(p, m, v, g, -1)
    assert e.value.code == 1
    with pytest.raises(nbm.NBMError) as e:
        prob.adam_step(p, m, v, g, 0, lr=0.0)
    assert e.value.code == 1
    with pytest.raises(nbm.NBMError) as e:
        prob.loss_grad_shard(p, 100, 90, 20)  # shard past the end of the batch
    assert e.value.code == 1
