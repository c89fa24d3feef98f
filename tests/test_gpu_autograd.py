"""Differentiation form: relaxed pilot p = tanh(theta), loss mean |H_hat - H_true|^2,
gradients from the library's adjoint kernels through torch.autograd -- checked against
the oracle's adjoint, a torch float64 autograd reference and central differences
(epsilon = 1e-3, loss accumulated in float64)."""
import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    import paper_2206_05506_gb300 as pk
    from paper_2206_05506_gb300.autograd import relaxed_estimate
    w = C.DIFFERENTIATION                     # M=64, N=1023, K=8, L=64, 64 frames
    bits, h, Y = C.make(w)
    rng = np.random.default_rng(99)
    theta = rng.standard_normal(w.N).astype(np.float32)
    return pk, relaxed_estimate, w, h, Y, theta


def _loss_and_grads(relaxed_estimate, w, h, Y, theta, dev):
    Yd = torch.from_numpy(Y).to(dev).requires_grad_(True)
    th = torch.from_numpy(theta).to(dev).requires_grad_(True)
    Ht = torch.from_numpy(h.astype(np.complex64)).to(dev)
    H = relaxed_estimate(Yd, th, w.K, w.L)
    loss = (H - Ht).abs().pow(2).mean()
    loss.backward()
    return H.detach(), loss.item(), Yd.grad, th.grad


def test_gradients_match_oracle_adjoint(case):
    pk, relaxed_estimate, w, h, Y, theta = case
    dev = torch.device("cuda", 0)
    H, loss, gY, gth = _loss_and_grads(relaxed_estimate, w, h, Y, theta, dev)
    p = np.tanh(theta.astype(np.float64))
    Href = O.estimate_real_pilot(Y, p, w.K, w.L)
    assert O.nmse(H.cpu().numpy(), Href) <= 1e-10
    G = 2 * (Href - h) / h.size                       # dLoss/dH for the mean |.|^2 loss
    dY, dp = O.adjoint(G, Y, p, w.K, w.L)
    assert O.nmse(gY.cpu().numpy(), dY) <= 1e-9
    assert O.nmse(gth.cpu().numpy(), dp * (1 - p ** 2)) <= 1e-9


def test_gradients_match_torch_autograd_reference(case):
    pk, relaxed_estimate, w, h, Y, theta = case
    dev = torch.device("cuda", 0)
    _, loss, gY, gth = _loss_and_grads(relaxed_estimate, w, h, Y, theta, dev)
    # float64 torch reference on the CPU: the forward written as a circulant product
    F, M, N = Y.shape
    Yt = torch.tensor(Y, dtype=torch.complex128, requires_grad=True)
    tt = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    idx = (torch.arange(N)[:, None] - torch.arange(w.K * w.L)[None, :]) % N
    P = torch.tanh(tt)[idx].to(torch.complex128)
    Hr = (Yt.reshape(F * M, N) @ P / N).reshape(F, M, w.K, w.L)
    lr = (Hr - torch.tensor(h)).abs().pow(2).mean()
    lr.backward()
    assert abs(loss - lr.item()) <= 1e-5 * lr.item()
    assert O.nmse(gY.cpu().numpy(), Yt.grad.numpy()) <= 1e-9
    assert O.nmse(gth.cpu().numpy(), tt.grad.numpy()) <= 1e-9


def test_central_differences(case):
    # directional central differences of the GPU forward (loss summed in float64)
    pk, relaxed_estimate, w, h, Y, theta = case
    dev = torch.device("cuda", 0)
    eps = 1e-3
    _, _, gY, gth = _loss_and_grads(relaxed_estimate, w, h, Y, theta, dev)
    Ht = torch.from_numpy(h).to(dev)

    def loss_at(Yv, thv):
        with torch.no_grad():
            H = relaxed_estimate(torch.from_numpy(Yv).to(dev), torch.from_numpy(thv).to(dev),
                                 w.K, w.L).to(torch.complex128)
            return (H - Ht).abs().pow(2).mean().item()

    rng = np.random.default_rng(5)
    gt = gth.cpu().numpy().astype(np.float64)
    g = gY.cpu().numpy().astype(np.complex128)
    for _ in range(3):
        # unit-variance directions, so eps * d stays far above the float32 spacing of the
        # perturbed arguments; the directional derivative is then ~ the gradient's norm
        d = rng.standard_normal(theta.size)
        fd = (loss_at(Y, (theta + eps * d).astype(np.float32)) -
              loss_at(Y, (theta - eps * d).astype(np.float32))) / (2 * eps)
        an = float(np.dot(gt, d))
        assert abs(fd - an) <= 2e-3 * abs(an) + 1e-4 * np.linalg.norm(gt)
        D = rng.standard_normal(Y.shape) + 1j * rng.standard_normal(Y.shape)
        fd = (loss_at((Y + eps * D).astype(np.complex64), theta) -
              loss_at((Y - eps * D).astype(np.complex64), theta)) / (2 * eps)
        an = float(np.sum(g.real * D.real + g.imag * D.imag))
        assert abs(fd - an) <= 2e-3 * abs(an) + 1e-4 * np.linalg.norm(g)


def test_one_optimisation_step_lowers_the_loss(case):
    # end-to-end pilot optimisation: a small gradient step on theta reduces the loss
    pk, relaxed_estimate, w, h, Y, theta = case
    dev = torch.device("cuda", 0)
    _, l0, _, gth = _loss_and_grads(relaxed_estimate, w, h, Y, theta, dev)
    th1 = theta - 0.5 * gth.cpu().numpy() / (np.linalg.norm(gth.cpu().numpy()) + 1e-30) * 1e-2
    _, l1, _, _ = _loss_and_grads(relaxed_estimate, w, h, Y, th1.astype(np.float32), dev)
    assert l1 < l0
