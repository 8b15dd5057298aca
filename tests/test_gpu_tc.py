"""GPU checks of the tensor-core (tcgen05) digit-plane contractions, through the step-level C ABI
(aci_k_frame_gemm_prec, aci_k_pi_block_prec) and aci_elementwise_ex with a BF16xS precision.

References are the definitions: the matrix product (numpy, FP64) and the CPU oracle of ACI. The
tolerance of a contraction is the a-priori bound of the exact digit split, computed here from the
inputs alone: with row scales 2^e_r > max|A[r,:]|, column scales 2^f_c > max|B[:,c]|, digits of b
bits (the largest b <= 7 with S K (2^b - 1)^2 < 2^24) and S digits,
    |C - AB| <= K 2^(e_r + f_c) 2^(-b S) (S + 3.1),
plus the FP64 rounding of the numpy reference (gamma_K |A||B|) and of the final recombination.
Integer-valued inputs whose digits are exact give the exact product, compared bit for bit.
"""

import numpy as np
import pytest

import oracle
from synthetic.fields import config_inputs
from synthetic.tt import tt_eval, tt_full, tt_random_uniform

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


def digit_bits(S, K2):
    b = 7
    while b > 2 and S * K2 * (2 ** b - 1) ** 2 >= 2 ** 24:
        b -= 1
    return b


def scale_exp(x, axis):
    """Smallest e with max|x| < 2^e along `axis` (0 for an all-zero line)."""
    m = np.abs(x).max(axis=axis)
    return np.where(m > 0, np.frexp(m)[1], 0).astype(np.float64)


def as_real(A, B):
    """The real forms the contraction runs: A'' (M x 2K), B'' (2K x 2N) for complex operands."""
    if not np.iscomplexobj(A):
        return A, B
    K, N = B.shape
    Ar = A.view(np.float64).reshape(A.shape[0], 2 * A.shape[1])
    Br = np.empty((2 * K, 2 * N))
    Br[0::2, 0::2], Br[0::2, 1::2] = B.real, B.imag
    Br[1::2, 0::2], Br[1::2, 1::2] = -B.imag, B.real
    return Ar, Br


def product_bound(A, B, S):
    """Per-entry bound of |C_split - A B| for the real forms (complex: per real and imaginary part)."""
    Ar, Br = as_real(A, B)
    K2 = Ar.shape[1]
    b = digit_bits(S, K2)
    er, fc = scale_exp(Ar, 1), scale_exp(Br, 0)
    split = K2 * np.exp2(er[:, None] + fc[None, :] - b * S) * (S + 3.1)
    gamma = 2 * K2 * 2.0 ** -53
    ref_round = gamma * (np.abs(Ar) @ np.abs(Br))
    Cr = Ar @ Br
    # + one rounding of the recombination, and subnormal products of the reference (absolute)
    bound = split + ref_round + 2.0 ** -51 * np.abs(Cr) + K2 * 2.0 ** -1074
    if np.iscomplexobj(A):
        bound = bound[:, 0::2] + 1j * bound[:, 1::2]
    return bound


def check_within(got, ref, bound):
    if np.iscomplexobj(ref):
        assert np.all(np.abs(got.real - ref.real) <= bound.real)
        assert np.all(np.abs(got.imag - ref.imag) <= bound.imag)
    else:
        err = np.abs(got - ref)
        assert np.all(err <= bound), (err / bound).max()


def rand_mat(rng, shape, cplx, spread=3.0):
    """Entries N(0,1) times per-row magnitudes 10^U(-spread, spread)."""
    x = rng.standard_normal(shape)
    if cplx:
        x = x + 1j * rng.standard_normal(shape)
    return x * 10.0 ** rng.uniform(-spread, spread, size=(shape[0], 1))


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("S", [2, 3, 4, 6, 8])
@pytest.mark.parametrize("shape", [(1, 1, 1), (37, 19, 53), (300, 70, 150), (257, 128, 129)])
def test_frame_gemm_digit_planes_within_bound(ctx, cplx, S, shape):
    M, K, N = shape
    rng = np.random.default_rng(M * 131 + N * 7 + S)
    A = rand_mat(rng, (M + 9, K + 3), cplx)
    B = np.ascontiguousarray(rand_mat(rng, (N + 5, K), cplx).T)  # column magnitudes spread too
    rows = rng.permutation(M + 9)[:M].astype(np.int32)
    cols = rng.permutation(N + 5)[:N].astype(np.int32)
    got = ctx.frame_gemm(dev(A), dev(B), dev(rows), dev(cols), K=K, precision=f"bf16x{S}").cpu().numpy()
    Ag, Bg = A[rows, :K], B[:K][:, cols]
    check_within(got, Ag @ Bg, product_bound(Ag, Bg, S))


@pytest.mark.parametrize("cplx", [False, True])
def test_frame_gemm_exact_on_integer_digits(ctx, cplx):
    """Integers below 2^7 with a 100 in every row and column are one exact digit each: the
    tensor-core product must equal the integer product exactly (every index and layout)."""
    rng = np.random.default_rng(5)
    M, K, N = 261, 77, 190
    A = rng.integers(-99, 100, size=(M, K)).astype(np.float64)
    B = rng.integers(-99, 100, size=(K, N)).astype(np.float64)
    A[:, 0] = 100.0
    B[0, :] = -100.0
    if cplx:
        A = A + 1j * rng.integers(-99, 100, size=(M, K))
        B = B + 1j * rng.integers(-99, 100, size=(K, N))
    for S in (2, 5):
        got = ctx.frame_gemm(dev(A), dev(B), precision=f"bf16x{S}").cpu().numpy()
        assert np.array_equal(got, A @ B)


def test_frame_gemm_special_values(ctx):
    """Zero lines give exact zeros, rows of 1e300 and 1e-300 keep their own scales, subnormal
    entries are split from their bits, and a NaN or Inf reaches every entry of its row and column."""
    rng = np.random.default_rng(9)
    M, K, N = 140, 40, 70
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    A[3] = 0.0
    A[4] *= 1e300
    A[5] *= 1e-300
    A[6] = 5e-310 * rng.standard_normal(K)
    got = ctx.frame_gemm(dev(A), dev(B), precision="bf16x8").cpu().numpy()
    ref = A @ B
    assert np.all(got[3] == 0.0)
    check_within(got, ref, product_bound(A, B, 8))
    A2 = A.copy()
    A2[7, 11] = np.nan
    B2 = B.copy()
    B2[13, 20] = np.inf
    got = ctx.frame_gemm(dev(A2), dev(B2), precision="bf16x8").cpu().numpy()
    assert np.all(np.isnan(got[7])) and np.all(np.isnan(got[:, 20]))
    mask = np.ones_like(got, dtype=bool)
    mask[7] = False
    mask[:, 20] = False
    assert np.all(np.isfinite(got[mask]))


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("S", [3, 6, 8])
@pytest.mark.parametrize("shape", [(24, 12, 13, 24), (300, 64, 48, 150), (512, 128, 128, 512)])
def test_pi_block_mul_within_bound(ctx, cplx, S, shape):
    M, K0, K1, N = shape
    rng = np.random.default_rng(M + N + S)
    A = [rand_mat(rng, (M, K0), cplx, 1.0), rand_mat(rng, (M, K1), cplx, 1.0)]
    B = [rand_mat(rng, (K0, N), cplx, 1.0), rand_mat(rng, (K1, N), cplx, 1.0)]
    Pi, mx = ctx.pi_block([dev(a) for a in A], [dev(b) for b in B], "mul", precision=f"bf16x{S}")
    Pi = Pi.cpu().numpy()
    p0, p1 = A[0] @ B[0], A[1] @ B[1]
    b0, b1 = product_bound(A[0], B[0], S), product_bound(A[1], B[1], S)
    if cplx:
        b0, b1 = np.abs(b0.real) + np.abs(b0.imag), np.abs(b1.real) + np.abs(b1.imag)
    # |(p0 + d0)(p1 + d1) - p0 p1| <= |p0| |d1| + |p1| |d0| + |d0| |d1|, plus one rounding of the product
    bound = np.abs(p0) * b1 + np.abs(p1) * b0 + b0 * b1 + 2.0 ** -50 * np.abs(p0 * p1)
    assert np.all(np.abs(Pi - p0 * p1) <= bound)
    assert abs(mx - np.abs(Pi).max()) <= 4e-16 * np.abs(Pi).max()


@pytest.mark.parametrize("op", ["mul_conj", "abs2_mul", "affine"])
def test_pi_block_ops_complex(ctx, op):
    rng = np.random.default_rng(17)
    M, K, N = 200, 40, 90
    coef = (0.5 - 1j, 2.0, -1.5 + 0.25j, 0.75j)
    A = [rand_mat(rng, (M, K), True, 0.5) for _ in range(2)]
    B = [rand_mat(rng, (K, N), True, 0.5) for _ in range(2)]
    n = 1 if op == "abs2_mul" else 2
    Pi, mx = ctx.pi_block([dev(a) for a in A[:n]], [dev(b) for b in B[:n]], op, coef=coef, precision="bf16x8")
    Pi = Pi.cpu().numpy()
    a, b = A[0] @ B[0], A[1] @ B[1]
    ref = {"mul_conj": a * np.conj(b), "abs2_mul": np.abs(a) ** 2 * a,
           "affine": coef[0] + coef[1] * a + coef[2] * b + coef[3] * a * b}[op]
    # 8 digits of 7 bits: entries of the products carry ~1e-15 relative error; f amplifies it a few times
    assert np.abs(Pi - ref).max() <= 1e-13 * np.abs(ref).max()
    assert abs(mx - np.abs(Pi).max()) <= 4e-16 * np.abs(Pi).max()


def test_precision_argument_checked(ctx):
    from paper_2604_00037_gb300.binding import AciError
    A = dev(np.ones((4, 4)))
    for bad in (1, 9, -1):
        with pytest.raises(AciError, match="ACI_E_ARG"):
            ctx.frame_gemm(A, A, precision=bad)


# ---------------------------------------------------------------- the whole method at BF16xS

def _dense_err(y, a, b):
    exact = tt_full(a) * tt_full(b)
    return np.abs(tt_full(y) - exact).max() / np.abs(exact).max()


@pytest.mark.parametrize("S", [5, 6, 8])
def test_config1_mixed_precision_against_oracle(ctx, S):
    """The 1D quantics workload (L=12, d=2, a*b, tol 1e-10): at S >= 5 digit planes the product
    stays within 1e-8 of the FP64 oracle's output and of the exact product."""
    p = config_inputs(1)
    a, b = p["inputs"]
    got, info = ctx.elementwise([dev(c) for c in a], [dev(c) for c in b], "mul", p["tol"], p["max_rank"],
                                precision=f"bf16x{S}", profile=True)
    y = [c.cpu().numpy() for c in got]
    ref = oracle.aci([a, b], "mul", p["tol"], p["max_rank"])
    yr, yt = tt_full(ref["Y"]), tt_full(y)
    assert np.abs(yt - yr).max() <= 1e-8 * np.abs(yr).max()
    assert _dense_err(y, a, b) <= 1e-8
    assert info["kernels"]["pi"]["tensor_flops"] > 0 and info["kernels"]["frame"]["tensor_flops"] > 0


@pytest.mark.parametrize("S", [2, 3, 4])
def test_config1_low_digit_counts_run(ctx, S):
    """Fewer digits trade accuracy for speed; the error stays near the contraction's precision."""
    p = config_inputs(1)
    a, b = p["inputs"]
    got, info = ctx.elementwise([dev(c) for c in a], [dev(c) for c in b], "mul", p["tol"], p["max_rank"],
                                precision=f"bf16x{S}")
    y = [c.cpu().numpy() for c in got]
    assert _dense_err(y, a, b) <= {2: 1e-2, 3: 1e-4, 4: 1e-6}[S]


@pytest.mark.parametrize("seed", range(3))
def test_random_complex_mixed_precision(ctx, seed):
    rng = np.random.default_rng(40 + seed)
    a = tt_random_uniform(rng, 6, 3, 4, dtype=np.complex128, low=-1, high=1)
    b = tt_random_uniform(rng, 6, 3, 4, dtype=np.complex128, low=-1, high=1)
    got, info = ctx.elementwise([dev(c) for c in a], [dev(c) for c in b], "mul_conj", 1e-12, 64,
                                precision="bf16x7")
    y = [c.cpu().numpy() for c in got]
    exact = tt_full(a) * np.conj(tt_full(b))
    assert np.abs(tt_full(y) - exact).max() <= 1e-9 * np.abs(exact).max()


def test_config2_mixed_precision_sampled_error(ctx):
    """The 2D interleaved workload (L=40, chi=128, a*b, tol 1e-10) at 6 digit planes: sampled
    relative error against the exact product <= 1e-8."""
    p = config_inputs(2, 128)
    a, b = p["inputs"]
    got, info = ctx.elementwise([dev(c) for c in a], [dev(c) for c in b], "mul", p["tol"], p["max_rank"],
                                precision="bf16x6")
    y = [c.cpu().numpy() for c in got]
    rng = np.random.default_rng(8)
    pts = rng.integers(0, 2, size=(20000, 40))
    yv, fv = tt_eval(y, pts), tt_eval(a, pts) * tt_eval(b, pts)
    assert np.abs(yv - fv).max() / np.abs(fv).max() <= 1e-8
    assert max(info["ranks"]) <= p["max_rank"]


@pytest.mark.parametrize("S", [4, 6])
def test_tuned_tile_width_keeps_accuracy(ctx, S):
    """aci_opts.autotune chooses the digit-plane contraction's output tile width (128 x 32 or 128 x 64)
    per shape class by timing both: the digits and their sums are the same either way, so the
    product meets the same bar against the oracle."""
    p = config_inputs(1)
    a, b = p["inputs"]
    ref = tt_full(oracle.aci([a, b], "mul", p["tol"], p["max_rank"])["Y"])
    for _ in range(2):  # the second call reuses the tuned table
        got, info = ctx.elementwise([dev(c) for c in a], [dev(c) for c in b], "mul", p["tol"], p["max_rank"],
                                    precision=f"bf16x{S}", autotune=True)
        y = [c.cpu().numpy() for c in got]
        bound = 1e-8 if S >= 5 else 1e-6
        assert np.abs(tt_full(y) - ref).max() <= bound * np.abs(ref).max()
