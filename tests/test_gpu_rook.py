"""GPU parity of the rook pivot search (aci_k_prrlu_rook, aci_elementwise_ex with ACI_PIVOT_ROOK)
against the CPU oracle's rook search (reading R11) on identical seeded inputs.

Integer outputs (pivot positions, ranks) must agree exactly up to the first step at which any of
the oracle's argmax decisions had a top-2 gap below 1e-12 of the matrix scale (a near-tie that
summation order can flip); FP64 outputs agree to the rounding of residuals divided by the pivot.
"""

import numpy as np
import pytest

import oracle
from synthetic.tt import tt_full, tt_random_uniform

from tests.test_gpu_kernels import _compare_prrlu

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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def graded(rng, m, n, cplx, decades=12):
    r = min(m, n)
    U = rng.standard_normal((m, r))
    V = rng.standard_normal((r, n))
    if cplx:
        U = U + 1j * rng.standard_normal(U.shape)
        V = V + 1j * rng.standard_normal(V.shape)
    return (U * (10.0 ** -np.linspace(0, decades, r))) @ V


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("shape,chimax,taurel", [
    ((1, 1), 4, 0.0), ((1, 9), 4, 0.0), ((13, 1), 4, 0.0), ((37, 53), 30, 0.0),
    ((37, 53), 100, 1e-3), ((128, 96), 64, 0.0), ((257, 300), 200, 1e-6), ((512, 512), 256, 1e-10),
    ((1024, 640), 128, 1e-8)])
def test_rook_prrlu_matches_oracle(ctx, cplx, shape, chimax, taurel):
    m, n = shape
    rng = np.random.default_rng(m * 1000 + n + 7)
    M = graded(rng, m, n, cplx)
    tau = taurel * np.abs(M).max()
    g = ctx.prrlu(dev(M), tau, chimax, mode="rook")
    f = oracle.ldu_rook(M, tau, chimax)
    _compare_prrlu(g, f, M)


def test_rook_prrlu_without_factors_and_degenerate(ctx):
    rng = np.random.default_rng(5)
    M = graded(rng, 70, 50, False)
    g = ctx.prrlu(dev(M), 1e-9 * np.abs(M).max(), 40, with_lu=False, mode="rook")
    f = oracle.ldu_rook(M, 1e-9 * np.abs(M).max(), 40)
    assert list(g["I"]) == list(f["I"]) and list(g["J"]) == list(f["J"])
    z = ctx.prrlu(dev(np.zeros((5, 7))), 0.0, 4, mode="rook")
    assert z["k"] == 1 and z["eps"] == 0.0 and z["D"][0] == 0.0
    assert (z["I"][0], z["J"][0]) == (0, 0)
    o = ctx.prrlu(dev(np.ones((6, 6))), 1e-14, 6, mode="rook")  # exact ties: lowest index, rank 1
    assert (o["I"][0], o["J"][0]) == (0, 0) and o["k"] == 1 and o["eps"] == 0.0


def test_rook_prrlu_large_complex_cross_interpolates(ctx):
    """A Pi-sized block of the fused d = 8 workload (2048 x 2048 complex, 256 pivots): the GPU
    factors reproduce M on the pivot cross and the residual there is the Schur complement."""
    rng = np.random.default_rng(9)
    m = n = 2048
    M = graded(rng, m, 300, True, decades=14) @ (rng.standard_normal((300, n)) / 20)
    tau = 1e-12 * np.abs(M).max()
    g = ctx.prrlu(dev(M), tau, 256, mode="rook")
    k = g["k"]
    assert k == 256
    A = g["L"] @ (g["D"][:, None] * g["U"])
    I, J = g["I"], g["J"]
    scale = np.abs(M).max()
    assert np.abs(A[I, :] - M[I, :]).max() <= 1e-9 * scale
    assert np.abs(A[:, J] - M[:, J]).max() <= 1e-9 * scale
    # every pivot is the largest residual of its column among the rows still unused (sampled steps)
    for p in (0, 1, 17, 128, 255):
        Ip, Jp = list(I[:p]), list(J[:p])
        R = M[:, J[p]] - (g["L"][:, :p] @ (g["D"][:p] * g["U"][:p, J[p]]))
        R[Ip] = 0
        assert np.abs(R[I[p]]) >= np.abs(R).max() * (1 - 1e-9)


def compare_aci(ctx, inputs, op, tol, max_rank, **kw):
    """Tie-aware whole-call parity in rook mode (tests/parity.py): pivots of every update until the
    oracle's first near-tie, values always."""
    from tests.parity import tie_aware_parity
    gk = dict(pivot_mode="rook")
    if "seed" in kw:
        gk["seed"] = kw["seed"]
    return tie_aware_parity(ctx, inputs, op, tol, max_rank, oracle_kw=dict(pivot_mode="rook", **kw), gpu_kw=gk)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("cplx", [False, True])
def test_rook_aci_matches_oracle(ctx, seed, cplx):
    rng = np.random.default_rng(300 + seed)
    L = int(rng.integers(2, 9))
    d = int(rng.choice([2, 3, 4]))
    chi = int(rng.integers(1, 6))
    dt = np.complex128 if cplx else np.float64
    a = tt_random_uniform(rng, L, d, chi, dtype=dt, low=-1, high=1)
    b = tt_random_uniform(rng, L, d, chi, dtype=dt, low=-1, high=1)
    y, info, ref, ties = compare_aci(ctx, [a, b], "mul", 1e-12, 64, seed=seed)
    exact = tt_full(a) * tt_full(b)
    assert np.abs(tt_full(y) - exact).max() <= 1e-9 * np.abs(exact).max()


def test_rook_aci_fused_d8_complex(ctx):
    rng = np.random.default_rng(31)
    a = tt_random_uniform(rng, 4, 8, 6, dtype=np.complex128, low=-1, high=1)
    y, info, ref, ties = compare_aci(ctx, [a], "abs2_mul", 1e-12, 200)
    A = tt_full(a)
    assert np.abs(tt_full(y) - np.abs(A) ** 2 * A).max() <= 1e-9 * np.abs(A).max() ** 3
