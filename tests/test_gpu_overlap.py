"""GPU checks of the overlapped sweep schedule (aci_opts.sweep_overlap): the frame half-products
and Pi blocks computed over every candidate row or column on a second stream, then gathered after
each pivot search. The schedule changes only the rounding of the contractions (their K splits),
so against the oracle it meets the same bar as the plain schedule (tests/parity.py): every pivot valid
against the oracle following it, identical ranks, iterations and final pivots, values within 1e-12
of max|y|. Local dimensions 3 and 4
(where the automatic choice keeps the plain schedule) are forced on; the degenerate lengths
L = 2 (one bond: nothing to overlap) and L = 3 (the shortest overlapped sweep) are included."""

import numpy as np
import pytest

from synthetic.tt import tt_full, tt_random_uniform

from tests.parity import followed_parity, to_dev, to_np

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


def run(ctx, inputs, op, tol, max_rank, overlap, **kw):
    ins = [to_dev(x) for x in inputs]
    if op == "abs2_mul":
        ins.append(None)
    return ctx.elementwise(*ins, op=op, tol=tol, max_rank=max_rank, pivots=True, overlap=overlap, **kw)


def check_vs_oracle(ctx, inputs, op, tol, max_rank, overlap="on", coef=None):
    """Followed parity (tests/parity.py) in the given schedule; returns (y, info, differ)."""
    y, info, ref = followed_parity(ctx, inputs, op, tol, max_rank, coef=coef, gpu_kw=dict(overlap=overlap))
    return y, info, ref["follow"]["differ"]


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("d", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_overlapped_matches_oracle(ctx, seed, d, cplx):
    rng = np.random.default_rng(700 + 10 * seed + d)
    L = int(rng.integers(3, 9))
    chi = int(rng.integers(1, 7))
    dt = np.complex128 if cplx else np.float64
    a = tt_random_uniform(rng, L, d, chi, dtype=dt, low=-1, high=1)
    b = tt_random_uniform(rng, L, d, chi, dtype=dt, low=-1, high=1)
    y, info, differ = check_vs_oracle(ctx, [a, b], "mul", 1e-12, 64)
    exact = tt_full(a) * tt_full(b)
    assert np.abs(tt_full(y) - exact).max() <= 1e-9 * np.abs(exact).max()


@pytest.mark.parametrize("op", ["mul_conj", "abs2_mul", "affine"])
def test_overlapped_ops_complex(ctx, op):
    rng = np.random.default_rng(41)
    a = tt_random_uniform(rng, 6, 2, 4, dtype=np.complex128, low=-1, high=1)
    b = tt_random_uniform(rng, 6, 2, 3, dtype=np.complex128, low=-1, high=1)
    coef = (0.5 - 1j, 2.0, -1.5 + 0.25j, 0.75j) if op == "affine" else None
    inputs = [a] if op == "abs2_mul" else [a, b]
    check_vs_oracle(ctx, inputs, op, 1e-12, 64, coef=coef)


@pytest.mark.parametrize("L", [2, 3])
def test_overlapped_short_chains(ctx, L):
    rng = np.random.default_rng(50 + L)
    a = tt_random_uniform(rng, L, 2, 2, dtype=np.float64, low=-1, high=1)
    b = tt_random_uniform(rng, L, 2, 3, dtype=np.float64, low=-1, high=1)
    y, info, differ = check_vs_oracle(ctx, [a, b], "mul", 1e-12, 64)
    assert differ == 0


def test_overlapped_agrees_with_plain_on_a_quantics_field(ctx):
    """A 2D quantics product (L = 16, d = 2, ranks up to 24): both schedules reach the same ranks
    and pivots and outputs equal to rounding."""
    from synthetic.fields import fourier_config2
    a, _ = fourier_config2(5, 24, nbits=8, nmodes=40)
    b, _ = fourier_config2(6, 24, nbits=8, nmodes=40)
    y1, i1 = run(ctx, [a, b], "mul", 1e-10, 48, "on")
    y0, i0 = run(ctx, [a, b], "mul", 1e-10, 48, "off")
    assert i1["ranks"] == i0["ranks"]
    assert i1["pivot_rows"] == i0["pivot_rows"] and i1["pivot_cols"] == i0["pivot_cols"]
    f1 = tt_full(to_np(y1))
    f0 = tt_full(to_np(y0))
    assert np.abs(f1 - f0).max() <= 1e-12 * np.abs(f0).max()


def test_overlapped_mixed_precision(ctx):
    rng = np.random.default_rng(77)
    a = tt_random_uniform(rng, 7, 2, 5, dtype=np.float64, low=-1, high=1)
    b = tt_random_uniform(rng, 7, 2, 4, dtype=np.float64, low=-1, high=1)
    got, info = run(ctx, [a, b], "mul", 1e-10, 64, "on", precision="bf16x6")
    exact = tt_full(a) * tt_full(b)
    assert np.abs(tt_full(to_np(got)) - exact).max() <= 1e-8 * np.abs(exact).max()


def test_bad_overlap_value_is_rejected(ctx):
    from paper_2604_00037_gb300 import binding
    from paper_2604_00037_gb300.binding import AciError
    rng = np.random.default_rng(3)
    a = to_dev(tt_random_uniform(rng, 4, 2, 2, dtype=np.float64, low=-1, high=1))
    saved = dict(binding.OVERLAP_MODES)
    binding.OVERLAP_MODES["bad"] = 7
    try:
        with pytest.raises(AciError) as e:
            ctx.elementwise(a, a, op="mul", overlap="bad")
        assert "ACI_E_ARG" in str(e.value)
    finally:
        binding.OVERLAP_MODES.clear()
        binding.OVERLAP_MODES.update(saved)
