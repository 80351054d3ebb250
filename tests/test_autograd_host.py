"""Host-side parts of the autograd wrapper that need no GPU: the stereo unary
log g = -beta * cost (Sec. 6's matching cost) and its chain rule to beta."""
import numpy as np
import torch

from paper_1010_0012_gb300 import autograd as ag


def test_unary_in_fp32_equals_the_fp64_product_rounded_once():
    """The product of two FP32 numbers is exact in FP64, so the FP32 multiply
    gives the FP64 product rounded to FP32 bit for bit."""
    cost = torch.from_numpy(np.random.default_rng(0).integers(0, 21, (40, 30, 16)).astype(np.float32))
    for b in (0.1, 0.37, 1.7, 3e-3):
        beta = torch.tensor(b, dtype=torch.float32)
        got = ag._NegScaledCost.apply(cost, beta)
        want = (-beta.double() * cost.double()).float()
        assert torch.equal(got, want)


def test_beta_gradient_is_the_fp64_sum():
    rng = np.random.default_rng(1)
    cost = torch.from_numpy(rng.integers(0, 21, (20, 25, 8)).astype(np.float32))
    beta = torch.tensor(0.25, dtype=torch.float32, requires_grad=True)
    g = torch.from_numpy(rng.standard_normal((20, 25, 8)).astype(np.float32))
    ag._NegScaledCost.apply(cost, beta).backward(g)
    want = -float((g.double() * cost.double()).sum())
    assert abs(float(beta.grad) - want) <= 1e-6 * abs(want)
