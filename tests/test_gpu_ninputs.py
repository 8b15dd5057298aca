"""f of more than two inputs (aci_elementwise_n): the product x^1 x^2 ... x^N of N = 3 and 4
tensor trains (Sec. 2.1 defines the method for N inputs; each input keeps its own frames and Pi
block, and f combines the N blocks entrywise). Followed parity against the oracle (tests/parity.py)
and the dense product."""

import numpy as np
import pytest

from synthetic import tt_full, tt_random_uniform
from tests.parity import followed_parity, to_dev

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


@pytest.mark.parametrize("N", [3, 4])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("overlap", ["off", "on"])
def test_product_of_n_inputs(ctx, N, cplx, overlap):
    rng = np.random.default_rng(10 * N + cplx)
    dt = np.complex128 if cplx else np.float64
    ins = [tt_random_uniform(rng, 7, 2, 2, dtype=dt, low=-1, high=1) for _ in range(N)]
    gk = dict(overlap=overlap)
    y, info = ctx.elementwise([to_dev(x) for x in ins], None, "mul", 1e-13, 64, pivots=True, history=True, **gk)
    y = [c.cpu().numpy() for c in y]
    y2, info2, ref = followed_parity(ctx, ins, "mul", 1e-13, 64, gpu=(y, info), gpu_kw=gk)
    exact = np.prod([tt_full(x) for x in ins], axis=0)
    assert np.abs(tt_full(y) - exact).max() <= 1e-11 * np.abs(exact).max()


def test_n_inputs_argument_errors(ctx):
    from paper_2604_00037_gb300.binding import AciError
    rng = np.random.default_rng(2)
    ins = [to_dev(tt_random_uniform(rng, 5, 2, 2, low=-1, high=1)) for _ in range(3)]
    with pytest.raises(AciError, match="ACI_E_ARG"):
        ctx.elementwise(ins, None, "affine", 1e-12, 16, coef=(1, 1, 1, 1))  # > 2 inputs: product only
    with pytest.raises(AciError, match="ACI_E_ARG"):
        ctx.elementwise(ins, None, "mul", 1e-12, 16, precision="bf16x6")   # > 2 inputs: FP64 only
    bad = ins[:2] + [to_dev(tt_random_uniform(rng, 6, 2, 2, low=-1, high=1))]
    with pytest.raises(AciError, match="ACI_E_SHAPE"):
        ctx.elementwise(bad, None, "mul", 1e-12, 16)
