"""GPU parity of the pivot-proposer network's kernels (aci_k_mlp_forward / _grad / _adam) with
the CPU reference oracle/mlp.py (float64), on seeded inputs. FP32 kernels against a float64
reference: logits agree to ~1e-5 relative, gradients to ~1e-4 relative (FP32 atomics in the sums
over samples), Adam to FP32 rounding."""

import numpy as np
import pytest

from oracle import mlp
from synthetic.weights import proposer_init

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_00037_gb300.binding import Context
    c = Context(0)
    yield c
    c.close()


def data(seed, n, F):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, F)).astype(np.float32)
    y = (X[:, 0] + 0.5 * X[:, min(1, F - 1)] ** 2 + 0.3 * rng.standard_normal(n) > 0.4).astype(np.float32)
    return X, y


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("n,F", [(1, 1), (17, 7), (1000, 7), (4099, 16)])
def test_forward_matches_reference(ctx, n, F):
    X, _ = data(n, n, F)
    p = proposer_init(n + F, F)
    assert ctx.mlp_param_count(F) == len(p)
    z = ctx.mlp_forward(cuda(X), cuda(p)).cpu().numpy()
    zr, _ = mlp.forward(p, X, F)
    assert np.abs(z - zr).max() <= 1e-5 * (1 + np.abs(zr).max())
    # FP16 weights: the reference with every weight rounded to FP16
    z16 = ctx.mlp_forward(cuda(X), cuda(p), fp16=True).cpu().numpy()
    zr16, _ = mlp.forward(p.astype(np.float16).astype(np.float32), X, F)
    assert np.abs(z16 - zr16).max() <= 1e-5 * (1 + np.abs(zr16).max())


@pytest.mark.parametrize("n,F,pw", [(5, 3, 1.0), (777, 7, 3.0), (20000, 9, 1.0)])
def test_gradient_matches_reference(ctx, n, F, pw):
    X, y = data(100 + n, n, F)
    p = proposer_init(7, F)
    loss, g = ctx.mlp_grad(cuda(X), cuda(y), cuda(p), pw)
    lr, gr = mlp.loss_grad(p, X, y, F, pw)
    assert loss == pytest.approx(lr, rel=1e-5)
    g = g.cpu().numpy()
    assert np.abs(g - gr).max() <= 1e-4 * np.abs(gr).max() + 1e-7


def test_adam_matches_reference(ctx):
    rng = np.random.default_rng(3)
    k = 5000
    p, g = rng.standard_normal(k).astype(np.float32), rng.standard_normal(k).astype(np.float32)
    m, v = (0.1 * rng.standard_normal(k)).astype(np.float32), rng.uniform(0, 0.1, k).astype(np.float32)
    P, G, Mt, V = cuda(p), cuda(g), cuda(m), cuda(v)
    ctx.mlp_adam(P, G, Mt, V, 7, 1e-3)
    pr, mr, vr = mlp.adam(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64), v.astype(np.float64), 7, 1e-3)
    assert np.abs(P.cpu().numpy() - pr).max() <= 1e-6
    assert np.abs(Mt.cpu().numpy() - mr).max() <= 1e-6 and np.abs(V.cpu().numpy() - vr).max() <= 1e-6


def test_training_reduces_the_loss(ctx):
    X, y = data(11, 8000, 6)
    Xd, yd = cuda(X), cuda(y)
    P = cuda(proposer_init(1, 6))
    Mt, V = torch.zeros_like(P), torch.zeros_like(P)
    first = None
    for t in range(1, 201):
        loss, g = ctx.mlp_grad(Xd, yd, P, 1.0)
        first = loss if first is None else first
        ctx.mlp_adam(P, g, Mt, V, t, 3e-3)
    last, _ = ctx.mlp_grad(Xd, yd, P, 1.0)
    assert last < 0.6 * first
    acc = ((ctx.mlp_forward(Xd, P).cpu().numpy() > 0) == (y > 0.5)).mean()
    assert acc > 0.85
