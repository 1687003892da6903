"""GPU tests of the tensor-core termination MLP against the FP64 reference
evaluated on the same FP16-rounded weights and inputs (oracle/mlp.py):
forward outputs, the accumulated gradient of the asymmetric loss, and the
Adam step, to relative L2 1e-3 (FP32 vs FP64 accumulation, and fp16
rounding boundaries of the hidden activations)."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2411_12440_gb300 import scenes
from paper_2411_12440_gb300.learned import TerminationMLP
from tests.gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu


def _setup(m, seed):
    p = scenes.random_mlp_params(seed)
    x, t = scenes.random_mlp_batch(m, seed + 1)
    net = TerminationMLP(p)
    return p, x, t, net


@pytest.mark.parametrize("m", [1, 15, 1000, 70_001])
def test_forward_matches_reference(m):
    p, x, t, net = _setup(m, 10)
    y = net.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref, _ = omlp.forward(x.astype(np.float64), p, fp16=True)
    got = y.cpu().numpy()
    assert rel_l2(got, ref) < 1e-3
    assert np.abs(got - ref).max() < 1e-2 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("m", [16, 127, 3001, 65_536])
def test_backward_matches_reference(m):
    p, x, t, net = _setup(m, 20)
    g, loss = net.grad_of(torch.from_numpy(x).cuda(), torch.from_numpy(t.astype(np.float32)).cuda(), 3.0)
    torch.cuda.synchronize()
    lref, gref = omlp.loss_and_grad(x.astype(np.float64), p, t.astype(np.float32).astype(np.float64), 3.0,
                                    fp16=True)
    assert float(loss.item()) == pytest.approx(lref, rel=1e-3)
    gg = g.cpu().numpy()
    bounds = list(omlp.OFF.values()) + [omlp.NPARAM]
    for name, a, b in zip(omlp.OFF, bounds[:-1], bounds[1:]):
        assert rel_l2(gg[a:b], gref[a:b]) < 1e-3, (name, rel_l2(gg[a:b], gref[a:b]))


def test_adam_step_matches_reference_and_refreshes_fp16():
    p, x, t, net = _setup(500, 30)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t.astype(np.float32)).cuda()
    m1 = np.zeros(omlp.NPARAM)
    m2 = np.zeros(omlp.NPARAM)
    master = net.master.cpu().numpy().astype(np.float64)
    for step in (1, 2, 3):
        g, _ = net.grad_of(xd, td, 2.0)
        gcpu = g.cpu().numpy().astype(np.float64)
        net.adam(lr=1e-3)
        torch.cuda.synchronize()
        master, m1, m2 = omlp.adam(step, 1e-3, 0.9, 0.999, 1e-8, master, gcpu, m1, m2)
        assert np.allclose(net.master.cpu().numpy(), master, rtol=1e-5, atol=1e-7)
    w1 = net.w1t.float().cpu().numpy()
    assert np.array_equal(w1, net.master[:64 * 48].cpu().numpy().astype(np.float16).astype(np.float32))


def test_training_reduces_the_loss():
    """A few hundred steps on a fixed random regression problem lower the loss."""
    p, x, t, net = _setup(4096, 40)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t.astype(np.float32)).cuda()
    first = float(net.train_step(xd, td, lr=3e-3).item())
    for _ in range(300):
        last = net.train_step(xd, td, lr=3e-3)
    assert float(last.item()) < 0.5 * first
