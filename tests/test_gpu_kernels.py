"""GPU parity of each hot-path step, through the step-level C ABI (include/aci_kernels.h),
against the CPU oracle on identical seeded inputs.

Tolerances: FP64 contractions of length K differ from the oracle only in summation order, so
entries agree to a few ulp of sum |a||b|; we require <= 1e-13 relative to max|C| (K <= 512).
Integer outputs (pivot positions, ranks) must agree exactly; where the oracle records a
top-2 gap below 1e-12 of the matrix scale (a near-tie) only the prefix before it is compared.
"""

import numpy as np
import pytest

import oracle
from oracle.rng import random_tt_counter

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


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("cplx", [False, True])
def test_tt_random_bit_exact(ctx, cplx):
    ranks, dims = [1, 3, 5, 4, 1], [2, 3, 8, 2]
    got = ctx.tt_random(12345, ranks, dims, complex_values=cplx)
    ref = random_tt_counter(12345, ranks, dims, cplx)
    for g, r in zip(got, ref):
        assert np.array_equal(g.cpu().numpy(), r)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("shape", [(1, 1, 1), (37, 19, 53), (64, 128, 96), (300, 7, 45)])
def test_frame_gemm_with_gathers(ctx, cplx, shape):
    M, K, N = shape
    rng = np.random.default_rng(M * 7 + N)
    A = rng.standard_normal((M + 11, K + 3))
    B = rng.standard_normal((K, N + 5))
    if cplx:
        A = A + 1j * rng.standard_normal(A.shape)
        B = B + 1j * rng.standard_normal(B.shape)
    rows = rng.permutation(M + 11)[:M].astype(np.int32)
    cols = rng.permutation(N + 5)[:N].astype(np.int32)
    got = ctx.frame_gemm(dev(A), dev(B), arows=dev(rows), bcols=dev(cols), K=K).cpu().numpy()
    ref = A[rows, :K] @ B[:, cols]
    assert rel(got, ref) <= 1e-13


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("op", ["mul", "mul_conj", "abs2_mul", "affine"])
def test_pi_block_ops(ctx, cplx, op):
    rng = np.random.default_rng(5)
    M, N = 70, 45
    Ks = [33, 17]
    As = [rng.standard_normal((M, k)) for k in Ks]
    Bs = [rng.standard_normal((k, N)) for k in Ks]
    if cplx:
        As = [a + 1j * rng.standard_normal(a.shape) for a in As]
        Bs = [b + 1j * rng.standard_normal(b.shape) for b in Bs]
    coef = (0.5 - 1j, 2.0, -1.5 + 0.25j, 0.75j) if cplx else (0.5, 2.0, -1.5, 0.75)
    n = 1 if op == "abs2_mul" else 2
    Pi, mx = ctx.pi_block([dev(a) for a in As[:n]], [dev(b) for b in Bs[:n]], op=op, coef=coef)
    prods = [a @ b for a, b in zip(As[:n], Bs[:n])]
    ref = oracle.apply_op(op, prods, coef)
    got = Pi.cpu().numpy()
    assert rel(got, ref) <= 1e-12
    assert abs(mx - oracle.magnitude(got).max()) == 0.0


def _compare_prrlu(g, f, M):
    scale = np.abs(M).max()
    kk = min(g["k"], f["k"])
    # exact pivot parity up to the first oracle near-tie
    gaps = (f["best"] - f["second"]) / max(scale, 1e-300)
    limit = len(gaps)
    near = np.nonzero(gaps < 1e-12)[0]
    if len(near):
        limit = int(near[0])
    same = min(kk, limit)
    assert list(g["I"][:same]) == list(f["I"][:same])
    assert list(g["J"][:same]) == list(f["J"][:same])
    if len(near) == 0:
        assert g["k"] == f["k"]
        assert abs(g["eps"] - f["eps"]) <= 1e-12 * scale
        np.testing.assert_allclose(g["D"], f["D"], atol=1e-12 * scale, rtol=1e-12)
        # L[:, p] and U[p, :] are residual entries divided by the pivot D_p: their rounding
        # error is about eps_mach * scale / |D_p| (large for the late, small pivots).
        bound = 1e-13 * scale / np.abs(f["D"]) + 1e-12
        assert (np.abs(g["L"] - f["L"]) <= bound[None, :]).all()
        assert (np.abs(g["U"] - f["U"]) <= bound[:, None]).all()


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("shape,chimax,taurel", [
    ((1, 1), 4, 0.0), ((1, 9), 4, 0.0), ((13, 1), 4, 0.0), ((37, 53), 30, 0.0),
    ((37, 53), 100, 1e-3), ((128, 96), 64, 0.0), ((257, 300), 200, 1e-6), ((512, 512), 256, 1e-10),
    # launch shapes of the other variants (capacity m x n decides): 128 x 96 and every complex
    # block up to 2^16 entries take the 2D register kernel, 257 x 300 and 512 x 512 real the 1D one,
    # 600 x 400 real prrlu_cluster_kernel (cluster path, too wide for either register kernel);
    # 700 x 700 real and every larger complex block take the cooperative grid prrlu_kernel
    ((128, 300), 128, 1e-8), ((600, 400), 300, 1e-10), ((700, 700), 350, 1e-10),
    # 160 x 400 real: the 1D register kernel with 5 of its 16 warps holding rows
    ((160, 400), 150, 1e-10)])
def test_prrlu_matches_oracle(ctx, cplx, shape, chimax, taurel):
    m, n = shape
    rng = np.random.default_rng(m * 1000 + n)
    # graded spectrum so the tolerance stop is exercised
    r = min(m, n)
    U = rng.standard_normal((m, r))
    V = rng.standard_normal((r, n))
    if cplx:
        U = U + 1j * rng.standard_normal(U.shape)
        V = V + 1j * rng.standard_normal(V.shape)
    M = (U * (10.0 ** -np.linspace(0, 12, r))) @ V
    tau = taurel * np.abs(M).max()
    g = ctx.prrlu(dev(M), tau, chimax)
    f = oracle.ldu(M, tau, chimax)
    _compare_prrlu(g, f, M)


def test_prrlu_degenerate(ctx):
    g = ctx.prrlu(dev(np.zeros((5, 7))), 0.0, 4)
    assert g["k"] == 1 and g["eps"] == 0.0 and g["D"][0] == 0.0
    assert (g["I"][0], g["J"][0]) == (0, 0)
    g = ctx.prrlu(dev(np.ones((6, 6))), 1e-14, 6)  # exact ties: lowest linear index, rank 1
    assert (g["I"][0], g["J"][0]) == (0, 0) and g["k"] == 1 and g["eps"] == 0.0


@pytest.mark.parametrize("cplx", [False, True])
def test_apply_pinv(ctx, cplx):
    rng = np.random.default_rng(9)
    M = rng.standard_normal((40, 30))
    if cplx:
        M = M + 1j * rng.standard_normal(M.shape)
    f = oracle.ldu(M, 0.0, 12)
    LI = f["L"][f["I"], :]
    UJ = f["U"][:, f["J"]]
    T = rng.standard_normal((25, 12)) + (1j * rng.standard_normal((25, 12)) if cplx else 0)
    got = ctx.apply_pinv(dev(T), dev(LI), dev(f["D"]), dev(UJ)).cpu().numpy()
    P = LI @ np.diag(f["D"]) @ UJ
    ref = np.linalg.solve(P.T, T.T).T
    assert rel(got, ref) <= 1e-10


def test_pivot_reciprocal_within_two_ulp(ctx):
    """The pivot search's reciprocal (approximate FP64 seed + two Newton-Raphson steps) against 1/x."""
    rng = np.random.default_rng(17)
    x = np.concatenate([rng.uniform(-1, 1, 4000) * 10.0 ** rng.uniform(-29, 29, 4000),
                        [1.0, -3.0, 0.1, 1e-200, -1e250, 1e-300]])
    y = ctx.reciprocal(dev(x)).cpu().numpy()
    ref = 1.0 / x
    ulp = np.spacing(np.abs(ref))
    assert (np.abs(y - ref) <= 2 * ulp).all()
