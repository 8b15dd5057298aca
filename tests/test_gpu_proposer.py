"""GPU checks of the learned proposer's use in the sweep (ACI_PIVOT_PROPOSED) and of its training
data. Plain full-candidate ACI stays the reference: keeping every candidate must reproduce it bit
for bit; a proposer trained with the library's own kernels on recorded pivots must leave the
result within the tolerance of the exact product, as the full right-to-left sweeps guarantee."""

import numpy as np
import pytest

from synthetic.weights import proposer_init
from synthetic.tt import tt_full, tt_random_uniform

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


def dev(tt):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in tt]


def pair(seed, L=10, d=2, chi=5, cplx=False):
    rng = np.random.default_rng(seed)
    dt = np.complex128 if cplx else np.float64
    return (tt_random_uniform(rng, L, d, chi, dtype=dt, low=-1, high=1),
            tt_random_uniform(rng, L, d, chi, dtype=dt, low=-1, high=1))


@pytest.mark.parametrize("cplx", [False, True])
def test_keeping_every_candidate_reproduces_plain_aci(ctx, cplx):
    a, b = pair(1, cplx=cplx)
    ref, rinfo = ctx.elementwise(dev(a), dev(b), "mul", 1e-12, 64)
    ctx.set_proposer(torch.from_numpy(proposer_init(0, 7)).cuda(), keep=1e6)
    got, info = ctx.elementwise(dev(a), dev(b), "mul", 1e-12, 64, pivot_mode="proposed")
    ctx.set_proposer(None)
    assert info["ranks"] == rinfo["ranks"] and info["iterations"] == rinfo["iterations"]
    assert all(torch.equal(x, y) for x, y in zip(got, ref))


def test_recording_gives_features_and_pivot_labels(ctx):
    a, b = pair(2)
    read = ctx.record_proposer_data(200000)
    _, info = ctx.elementwise(dev(a), dev(b), "mul", 1e-12, 64)
    X, y, n = read()
    X, y = X.cpu().numpy(), y.cpu().numpy()
    assert n == len(y) > 0 and X.shape[1] == 7
    assert set(np.unique(y)) <= {0.0, 1.0} and 0 < y.mean() < 1
    assert np.all(X[:, 0] <= 0) and np.all(X[:, 0] >= -2) and np.all((X[:, 6] == 0) | (X[:, 6] == 1))
    # every iteration's left-to-right sweep labels k pivot rows and k pivot columns per bond
    assert y.sum() % 2 == 0


def test_trained_proposer_keeps_the_error(ctx):
    """Train on the pivots of plain ACI for a few products, then run held-out products with the
    learned restriction: the error against the exact product stays at the tolerance level."""
    read = ctx.record_proposer_data(400000)
    for s in range(6):
        a, b = pair(10 + s, L=10, d=2, chi=6)
        ctx.elementwise(dev(a), dev(b), "mul", 1e-10, 64)
    X, y, _ = read()
    P = torch.from_numpy(proposer_init(3, 7)).cuda()
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    pw = float((1 - y.mean()) / max(y.mean(), 1e-6))
    l0 = None
    for t in range(1, 301):
        loss, g = ctx.mlp_grad(X, y, P, pw)
        l0 = loss if l0 is None else l0
        ctx.mlp_adam(P, g, M, V, t, 2e-3)
    assert loss < l0
    ctx.set_proposer(P, keep=1.25)
    for s in range(3):
        a, b = pair(100 + s, L=10, d=2, chi=6)
        got, info = ctx.elementwise(dev(a), dev(b), "mul", 1e-10, 64, pivot_mode="proposed")
        exact = tt_full(a) * tt_full(b)
        y_ = tt_full([c.cpu().numpy() for c in got])
        assert np.abs(y_ - exact).max() <= 1e-8 * np.abs(exact).max()
    ctx.set_proposer(None)
