"""FP32 / complex64 inputs (ACI_R32 / ACI_C64: widened to FP64 / complex128 on load by the
library) and the batched workload with its FP32 pairs, every product checked against the oracle.

The oracle receives the same values widened to float64 / complex128 (exact), so the bar is that
of FP64 inputs: the followed parity of tests/parity.py for single calls (every pivot valid,
identical ranks, iterations and final pivots, values within 1e-12 of max|y|); in a batch, whose
results the C ABI returns without pivot histories, ranks and iteration counts must equal the
oracle's and values agree within 1e-12 of max|y| unless the oracle saw a near-tie (then within
10 x tol, as several results are correct)."""

import numpy as np
import pytest

import oracle
from synthetic import tt_eval, tt_full, tt_random_uniform
from synthetic.fields import batch_config4_pair, batch_config4_spec
from tests.parity import NEAR_TIE, followed_parity

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


def _f32(tt, cplx):
    return [c.astype(np.complex64 if cplx else np.float32) for c in tt]


def _wide(tt):
    return [c.astype(np.complex128 if np.iscomplexobj(c) else np.float64) for c in tt]


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("memory", ["device", "host"])
def test_fp32_inputs_match_the_oracle_on_their_values(ctx, cplx, memory):
    rng = np.random.default_rng(40 + cplx)
    dt = np.complex128 if cplx else np.float64
    a = _f32(tt_random_uniform(rng, 7, 2, 5, dtype=dt, low=-1, high=1), cplx)
    b = _f32(tt_random_uniform(rng, 7, 2, 4, dtype=dt, low=-1, high=1), cplx)
    op = "mul_conj" if cplx else "mul"
    if memory == "device":
        y, info, ref = followed_parity(ctx, [_wide(a), _wide(b)], op, 1e-12, 64)
        # the same call handed the FP32 cores: the library widens them, so everything is identical
        from tests.parity import to_dev
        yf, infof = ctx.elementwise(to_dev(a), to_dev(b), op=op, tol=1e-12, max_rank=64, pivots=True)
        assert infof["ranks"] == info["ranks"] and infof["pivot_rows"] == info["pivot_rows"]
        assert all(np.array_equal(c1.cpu().numpy(), c2) for c1, c2 in zip(yf, y))
        assert yf[0].dtype == (torch.complex128 if cplx else torch.float64)
    else:
        yh, infoh = ctx.elementwise(a, b, op=op, tol=1e-12, max_rank=64, out_memory="host")
        ref = oracle.aci([_wide(a), _wide(b)], op, 1e-12, 64)
        assert infoh["ranks"] == ref["ranks"]
        yr = tt_full(ref["Y"])
        assert np.abs(tt_full(yh) - yr).max() <= 1e-12 * np.abs(yr).max()


def test_mixed_dtypes_are_rejected(ctx):
    from paper_2604_00037_gb300.binding import AciError
    from tests.parity import to_dev
    rng = np.random.default_rng(3)
    a = tt_random_uniform(rng, 4, 2, 2, low=-1, high=1)
    with pytest.raises(AciError, match="ACI_E_DTYPE"):
        ctx.elementwise(to_dev(_f32(a, False)), to_dev(a), op="mul")


def _tie_aware(y, info, ref, tol, pts):
    ties = any(len(e["best"]) and ((e["best"] - e["second"]) / e["S"]).min() < NEAR_TIE for e in ref["log"])
    yv, rv = tt_eval(y, pts), tt_eval(ref["Y"], pts)
    scale = np.abs(rv).max()
    if not ties:
        assert info["ranks"] == ref["ranks"] and info["iterations"] == ref["iterations"]
        assert np.abs(yv - rv).max() <= 1e-12 * scale
    else:
        assert np.abs(yv - rv).max() <= 10 * tol * scale
    return ties


def _small_cfg4(n):
    """The n pairs of the batched workload (200-mode fields, FP32 odd pairs) with the lowest ranks,
    so that the oracle finishes each in seconds."""
    spec = sorted(batch_config4_spec(), key=lambda s: (s["chi"], s["nbits"]))[:n]
    return spec, [batch_config4_pair(s) for s in spec]


def test_batched_workload_every_product_matches_the_oracle(ctx):
    spec, pairs = _small_cfg4(6)
    assert {s["dtype"] for s in spec} == {"f32", "f64"} and {s["op"] for s in spec} == {"mul", "mul_conj"}
    items = []
    for s, (a, b) in zip(spec, pairs):
        dt = torch.float32 if s["dtype"] == "f32" else torch.float64
        items.append(dict(a=[torch.from_numpy(c).to(dt).cuda() for c in a], b=[torch.from_numpy(c).to(dt).cuda() for c in b],
                          op=s["op"], tol=s["tol"], max_rank=s["max_rank"]))
    res = ctx.elementwise_batch(items, streams=3)
    rng = np.random.default_rng(5)
    for s, (a, b), (cores, info) in zip(spec, pairs, res):
        assert info["status"] in ("ACI_OK", "ACI_W_NOT_CONVERGED")
        if s["dtype"] == "f32":  # the oracle sees the values the library was handed
            a, b = _wide(_f32(a, False)), _wide(_f32(b, False))
        ref = oracle.aci([a, b], s["op"], s["tol"], s["max_rank"], record=True)
        pts = rng.integers(0, 2, size=(4000, len(a)))
        _tie_aware([c.cpu().numpy() for c in cores], info, ref, s["tol"], pts)


def test_batched_workload_conj_on_a_complex_copy(ctx):
    """a * conj(b) is a * b for real fields; on a complex copy with b turned by exp(i pi / 3) the
    conjugation does real work (the exact product is a * b * exp(-i pi / 3))."""
    spec, pairs = _small_cfg4(3)
    rot = np.exp(1j * np.pi / 3)
    items, ins = [], []
    for s, (a, b) in zip(spec, pairs):
        ac = [c.astype(np.complex128) for c in a]
        bc = [c.astype(np.complex128) for c in b]
        bc[0] = bc[0] * rot
        ins.append((ac, bc))
        items.append(dict(a=[torch.from_numpy(c).cuda() for c in ac], b=[torch.from_numpy(c).cuda() for c in bc],
                          op="mul_conj", tol=s["tol"], max_rank=s["max_rank"]))
    res = ctx.elementwise_batch(items, streams=3)
    rng = np.random.default_rng(6)
    for s, (ac, bc), (cores, info) in zip(spec, ins, res):
        y = [c.cpu().numpy() for c in cores]
        ref = oracle.aci([ac, bc], "mul_conj", s["tol"], s["max_rank"], record=True)
        pts = rng.integers(0, 2, size=(4000, len(ac)))
        _tie_aware(y, info, ref, s["tol"], pts)
