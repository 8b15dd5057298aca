"""GPU checks of aci_elementwise_batch: independent products run concurrently on worker streams
must give exactly what aci_elementwise_ex gives for each product alone (same kernels, same
deterministic reductions), whatever the number of streams; a failing product reports its own
status without disturbing the others. Every product of a batch is also compared with the oracle
(here, and for the batched workload's own pairs in test_gpu_dtypes.py)."""

import numpy as np
import pytest

import oracle
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


def make_items(seed, n):
    """Uneven products: lengths 3-9, local dimensions 2-4, ranks 1-6, real and complex, several ops."""
    rng = np.random.default_rng(seed)
    items = []
    for i in range(n):
        L = int(rng.integers(3, 10))
        d = int(rng.choice([2, 3, 4]))
        cplx = bool(i % 3 == 2)
        dt = np.complex128 if cplx else np.float64
        a = tt_random_uniform(rng, L, d, int(rng.integers(1, 7)), dtype=dt, low=-1, high=1)
        b = tt_random_uniform(rng, L, d, int(rng.integers(1, 7)), dtype=dt, low=-1, high=1)
        op = ["mul", "mul_conj", "abs2_mul"][i % 3] if cplx else "mul"
        items.append(dict(a=a, b=None if op == "abs2_mul" else b, op=op, tol=1e-12, max_rank=64))
    return items


def same(x, y):
    return len(x) == len(y) and all(torch.equal(p, q) for p, q in zip(x, y))


@pytest.mark.parametrize("streams,overlap", [(1, "auto"), (3, "auto"), (0, "auto"), (3, "on")])
def test_batch_equals_single_calls(ctx, streams, overlap):
    """In a batch the automatic schedule is the plain one; an explicit schedule is kept."""
    items = make_items(1, 9)
    res = ctx.elementwise_batch([dict(it, a=dev(it["a"]), b=dev(it["b"]) if it["b"] is not None else None)
                                 for it in items], streams=streams, overlap=overlap)
    single = "off" if overlap == "auto" else overlap
    for it, (cores, info) in zip(items, res):
        assert info["status"] in ("ACI_OK", "ACI_W_NOT_CONVERGED")
        ins = [dev(it["a"])] + ([dev(it["b"])] if it["b"] is not None else [None])
        ref, rinfo = ctx.elementwise(*ins, op=it["op"], tol=it["tol"], max_rank=it["max_rank"], overlap=single)
        assert same(cores, ref)
        assert info["ranks"] == rinfo["ranks"] and info["iterations"] == rinfo["iterations"]


def test_batch_products_match_oracle_and_exact(ctx):
    items = make_items(2, 4)
    res = ctx.elementwise_batch([dict(it, a=dev(it["a"]), b=dev(it["b"]) if it["b"] is not None else None)
                                 for it in items], streams=4)
    for it, (cores, info) in zip(items, res):  # every product against the oracle
        ins = [it["a"]] + ([it["b"]] if it["b"] is not None else [])
        ref = oracle.aci(ins, it["op"], it["tol"], it["max_rank"])
        y = tt_full([c.cpu().numpy() for c in cores])
        assert info["ranks"] == ref["ranks"]
        assert np.abs(y - tt_full(ref["Y"])).max() <= 1e-12 * np.abs(tt_full(ref["Y"])).max()
    for it, (cores, info) in zip(items, res):
        A = tt_full(it["a"])
        B = tt_full(it["b"]) if it["b"] is not None else None
        exact = {"mul": lambda: A * B, "mul_conj": lambda: A * np.conj(B), "abs2_mul": lambda: np.abs(A) ** 2 * A}[it["op"]]()
        got = tt_full([c.cpu().numpy() for c in cores])
        assert np.abs(got - exact).max() <= 1e-9 * np.abs(exact).max()


def test_batch_reports_a_failing_product_alone(ctx):
    items = make_items(3, 5)
    bad = dict(items[2], max_rank=0)  # invalid: max_rank must be >= 1
    batch = [dict(it, a=dev(it["a"]), b=dev(it["b"]) if it["b"] is not None else None) for it in items]
    batch[2] = dict(bad, a=dev(bad["a"]), b=dev(bad["b"]) if bad["b"] is not None else None)
    res = ctx.elementwise_batch(batch, streams=2)
    assert res[2][1]["status"] == "ACI_E_ARG" and res[2][0] is None
    for i in (0, 1, 3, 4):
        assert res[i][1]["status"] in ("ACI_OK", "ACI_W_NOT_CONVERGED") and res[i][0] is not None


def test_batch_empty_and_host_outputs(ctx):
    assert ctx.elementwise_batch([]) == []
    items = make_items(4, 3)
    res = ctx.elementwise_batch([dict(it, a=dev(it["a"]), b=dev(it["b"]) if it["b"] is not None else None)
                                 for it in items], out_memory="host", streams=2)
    for it, (cores, info) in zip(items, res):
        assert isinstance(cores[0], np.ndarray)


def test_autotuned_concurrency_keeps_results(ctx):
    """batch_streams = 0 tries several concurrency levels on successive calls (then keeps the
    fastest); every call returns the same products."""
    items = make_items(5, 6)
    batch = [dict(it, a=dev(it["a"]), b=dev(it["b"]) if it["b"] is not None else None) for it in items]
    first = ctx.elementwise_batch(batch, streams=0)
    for _ in range(4):
        again = ctx.elementwise_batch(batch, streams=0)
        for (c1, i1), (c2, i2) in zip(first, again):
            assert same(c1, c2) and i1["ranks"] == i2["ranks"]


def test_contraction_tuner_keeps_parity(ctx):
    """aci_opts.autotune times the FP64 contractions' split-K granularity per shape class and keeps
    the fastest in the context: only the summation order of the contractions changes, so the
    products still meet the followed-parity bar against the oracle, alone and in a batch."""
    from tests.parity import followed_parity
    rng = np.random.default_rng(12)
    a = tt_random_uniform(rng, 8, 2, 5, low=-1, high=1)
    b = tt_random_uniform(rng, 8, 2, 4, low=-1, high=1)
    for _ in range(2):  # the second call reuses the tuned table
        followed_parity(ctx, [a, b], "mul", 1e-12, 64, gpu_kw=dict(autotune=True))
    items = make_items(6, 5)
    res = ctx.elementwise_batch([dict(it, a=dev(it["a"]), b=dev(it["b"]) if it["b"] is not None else None)
                                 for it in items], streams=3, autotune=True)
    for it, (cores, info) in zip(items, res):
        ins = [it["a"]] + ([it["b"]] if it["b"] is not None else [])
        ref = oracle.aci(ins, it["op"], it["tol"], it["max_rank"])
        y = tt_full([c.cpu().numpy() for c in cores])
        assert np.abs(y - tt_full(ref["Y"])).max() <= 1e-10 * np.abs(tt_full(ref["Y"])).max()
