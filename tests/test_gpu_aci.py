"""GPU parity of the whole ACI call (aci_elementwise_ex through the C ABI) against the oracle.

Bar (FP64), through tests/parity.py: the oracle follows the GPU's recorded pivots wherever they
are as valid as its own (every pivot of every update is checked against the oracle's Schur
complement), ranks, iteration counts and final pivots are identical, and output values agree
within 1e-12 of max|y| on every grid point (dense for small L) or on seeded samples. The
benchmarked sizes are covered by tests/test_gpu_fullsize.py.
"""

import numpy as np
import pytest

from synthetic import (config_inputs, tt_full, tt_eval, tt_random_uniform, random_tt_pair)
from tests.parity import followed_parity, to_dev, to_np
from synthetic.fields import exp_mode_tt, _site_angles

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


def compare_with_oracle(ctx, inputs, op, tol, max_rank, coef=None, dense=True, **kw):
    """GPU run with its pivot history, then the oracle following it (tests/parity.py): every
    pivot valid, identical ranks / iterations / final pivots, values within 1e-12 of max|y|."""
    gpu_kw = {k: v for k, v in kw.items() if k in ("overlap", "precision", "max_sweeps")}
    oracle_kw = {k: v for k, v in kw.items() if k not in gpu_kw}
    gk = dict(gpu_kw)
    if "seed" in oracle_kw:
        gk["seed"] = oracle_kw["seed"]
    if "init" in oracle_kw:
        gk["init"] = to_dev(oracle_kw["init"])
    y, info, ref = followed_parity(ctx, inputs, op, tol, max_rank, coef=coef, oracle_kw=oracle_kw, gpu_kw=gk,
                                   points=None if dense else np.random.default_rng(7).integers(
                                       0, inputs[0][0].shape[1], size=(20000, len(inputs[0]))))
    return y, info, ref, ref["follow"]["differ"]


def test_config1_parity(ctx):
    p = config_inputs(1)
    a, b = p["inputs"]
    y, info, ref, differ = compare_with_oracle(ctx, [a, b], "mul", p["tol"], p["max_rank"])
    assert differ == 0  # no near-tie on this workload: the GPU took the oracle's own pivots
    exact = tt_full(a) * tt_full(b)
    assert np.abs(tt_full(y) - exact).max() <= 10 * p["tol"] * np.abs(exact).max()
    assert info["kernel_launches"] > 0


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("cplx", [False, True])
def test_random_small_parity(ctx, seed, cplx):
    rng = np.random.default_rng(seed)
    L = int(rng.integers(2, 9))
    d = int(rng.choice([2, 3, 4]))
    chi = int(rng.integers(1, 6))
    dt = np.complex128 if cplx else np.float64
    a = tt_random_uniform(rng, L, d, chi, dtype=dt, low=-1, high=1)
    b = tt_random_uniform(rng, L, d, chi, dtype=dt, low=-1, high=1)
    compare_with_oracle(ctx, [a, b], "mul", 1e-12, 64, seed=seed)


@pytest.mark.parametrize("op", ["mul", "mul_conj", "abs2_mul", "affine"])
def test_ops_complex_parity(ctx, op):
    rng = np.random.default_rng(21)
    a = tt_random_uniform(rng, 7, 2, 3, dtype=np.complex128, low=-1, high=1)
    b = tt_random_uniform(rng, 7, 2, 3, dtype=np.complex128, low=-1, high=1)
    coef = (0.5 - 1j, 2.0, -1.5 + 0.25j, 0.75j)
    ins = [a] if op == "abs2_mul" else [a, b]
    y, info, ref, differ = compare_with_oracle(ctx, ins, op, 1e-13, 128, coef=coef)
    A, B = tt_full(a), tt_full(b)
    exact = {"mul": A * B, "mul_conj": A * np.conj(B), "abs2_mul": np.abs(A) ** 2 * A,
             "affine": coef[0] + coef[1] * A + coef[2] * B + coef[3] * A * B}[op]
    assert np.abs(tt_full(y) - exact).max() <= 1e-10 * np.abs(exact).max()


def test_fused_d8_ragged(ctx):
    rng = np.random.default_rng(3)
    a = tt_random_uniform(rng, 4, 8, 5, low=-1, high=1)
    b = tt_random_uniform(rng, 4, 8, 3, low=-1, high=1)
    compare_with_oracle(ctx, [a, b], "mul", 1e-12, 200)


def test_assembly_above_rank_256_capacity(ctx):
    """The output assembly takes one warp per row up to rank capacity 256 (8 columns per lane) and
    one thread per row above it: 18 sites of d = 2 with max_rank 300 give capacity 300 at the
    middle bonds, so the second form runs; against the oracle on 20000 points."""
    rng = np.random.default_rng(31)
    a = tt_random_uniform(rng, 18, 2, 4, low=-1, high=1)
    b = tt_random_uniform(rng, 18, 2, 3, low=-1, high=1)
    compare_with_oracle(ctx, [a, b], "mul", 1e-12, 300, dense=False)


def test_edge_cases(ctx):
    # L = 1: y = f(x) exactly
    a = [np.array([[[1.5], [-2.0], [0.25]]])]
    b = [np.array([[[2.0], [3.0], [-4.0]]])]
    got, info = ctx.elementwise(to_dev(a), to_dev(b), "mul", 1e-12, 4)
    assert np.array_equal(got[0].cpu().numpy(), a[0] * b[0])
    # L = 2, max_rank 1, and a zero input (Pi = 0 everywhere: rank 1, y = 0)
    rng = np.random.default_rng(0)
    a = tt_random_uniform(rng, 2, 2, 2, low=-1, high=1)
    z = [np.zeros_like(c) for c in a]
    compare_with_oracle(ctx, [a, a], "mul", 1e-12, 1)
    got, info = ctx.elementwise(to_dev(a), to_dev(z), "mul", 1e-12, 8)
    assert np.abs(tt_full(to_np(got))).max() == 0.0
    assert max(info["ranks"]) == 1


def test_single_modes_rank_one(ctx):
    L = 16
    a = exp_mode_tt(0.7 - 0.2j, _site_angles([5], L, 1, "1d", 2 * np.pi))
    b = exp_mode_tt(1.1 + 0.4j, _site_angles([-3], L, 1, "1d", 2 * np.pi))
    got, info = ctx.elementwise(to_dev(a), to_dev(b), "mul", 1e-12, 16)
    assert max(info["ranks"]) == 1
    x = np.arange(2 ** L) / 2 ** L
    exact = (0.7 - 0.2j) * (1.1 + 0.4j) * np.exp(2j * np.pi * 2 * x)
    assert np.abs(tt_full(to_np(got)) - exact).max() <= 1e-13


def test_host_memory_path_matches_device(ctx):
    p = config_inputs(1)
    a, b = p["inputs"]
    yd, _ = ctx.elementwise(to_dev(a), to_dev(b), "mul", p["tol"], p["max_rank"])
    yh, _ = ctx.elementwise(a, b, "mul", p["tol"], p["max_rank"], out_memory="host")
    for c1, c2 in zip(to_np(yd), yh):
        assert np.array_equal(c1, c2)


def test_warm_start_matches_oracle(ctx):
    p = config_inputs(1)
    a, b = p["inputs"]
    y0, _ = ctx.elementwise(to_dev(a), to_dev(b), "mul", p["tol"], p["max_rank"])
    init = to_np(y0)
    compare_with_oracle(ctx, [a, b], "mul", p["tol"], p["max_rank"], init=init)


def test_errors_are_reported(ctx):
    from paper_2604_00037_gb300.binding import AciError
    p = config_inputs(1)
    a, b = p["inputs"]
    with pytest.raises(AciError, match="ACI_E_SHAPE"):
        ctx.elementwise(to_dev(a), to_dev(b[:-1] + [np.ones((b[-1].shape[0], 2, 1))[:, :1]]), "mul", 1e-10, 8)
    with pytest.raises(AciError, match="ACI_E_ARG"):
        ctx.elementwise(to_dev(a), to_dev(b), "mul", -1.0, 8)
    with pytest.raises(AciError, match="ACI_E_DTYPE"):
        ctx.elementwise(to_dev(a), to_dev(b), "affine", 1e-10, 8, coef=(1j, 0, 0, 0))


@pytest.mark.parametrize("chi", [64, 128])
def test_config2_full_size_properties(ctx, chi):
    """The benchmarked workload (2D interleaved L=40, FP64, a*b, tol 1e-10, max_rank 2 chi):
    sampled error against the exact product and the interpolation property on J_1."""
    p = config_inputs(2, chi)
    a, b = p["inputs"]
    got, info = ctx.elementwise(to_dev(a), to_dev(b), "mul", p["tol"], p["max_rank"], pivots=True)
    y = to_np(got)
    rng = np.random.default_rng(7)
    pts = rng.integers(0, 2, size=(20000, 40))
    yv, fv = tt_eval(y, pts), tt_eval(a, pts) * tt_eval(b, pts)
    err = np.abs(yv - fv).max() / np.abs(fv).max()
    # the error estimate of the last sweep bounds the sampled error (heuristic, Sec. 2.6)
    assert err <= 20 * info["max_eps"] / info["scale"] + 1e-12, (err, info["max_eps"] / info["scale"])
    assert max(info["ranks"]) <= p["max_rank"]
