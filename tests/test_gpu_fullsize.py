"""Parity at the sizes the benchmark runs, and whole calls through every pivot-search variant.

The benchmarked workload is config 2 (2D interleaved quantics TTs, L = 40, d = 2, FP64 Fourier
fields with 200 modes, a*b, tol 1e-10 relative, max_rank 2 chi) at chi = 64 and 128: Pi blocks up
to 480 x 480, pivot searches in the 16-CTA register kernel, split-K contractions of 480 x 246 x 128
and the overlapped schedule's gathers at full size. Each call runs with its pivot history
recorded; the oracle then runs the same product following the GPU's pivots wherever they are as
valid as its own (tests/parity.py), which checks every pivot of every local update of all 20
sweeps against the oracle's own Schur complement, and the outputs are compared on 20000 seeded
grid points at 1e-12 of max|y|. Both schedules (overlapped and plain) are covered.

The other cases run whole calls whose block capacities select the pivot-search variants that the
benchmark does not reach: the shared-memory cluster kernel (a 600 x 400 real block; an 8 x 320
complex block of a fused d = 8 chain) and the cooperative grid kernel (a 700 x 700 real block; a
512 x 512 complex block of a d = 8 chain of length 6).
"""

import numpy as np
import pytest

from synthetic import config_inputs, tt_eval, tt_full
from tests.parity import followed_parity, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

_followed = {}  # (chi, pivot history) -> followed oracle run, shared by the two schedules


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_00037_gb300.binding import Context
    c = Context(0)
    yield c
    c.close()


def _history_key(info):
    return tuple(sorted((k, tuple(v[0]), tuple(v[1])) for k, v in info["history"].items()))


@pytest.mark.parametrize("chi", [64, 128])
@pytest.mark.parametrize("overlap", ["on", "off"])
def test_config2_followed_parity(ctx, chi, overlap):
    p = config_inputs(2, chi)
    a, b = p["inputs"]
    pts = np.random.default_rng(7).integers(0, 2, size=(20000, len(a)))
    gpu = run_gpu(ctx, [a, b], "mul", p["tol"], p["max_rank"], overlap=overlap)
    key = (chi, _history_key(gpu[1]))
    if key in _followed:  # the other schedule chose the same pivots: the followed run is the same
        y, info = gpu
        ref = _followed[key]
        yv, rv = tt_eval(y, pts), tt_eval(ref["Y"], pts)
        assert np.abs(yv - rv).max() <= 1e-12 * np.abs(rv).max()
        assert info["ranks"] == ref["ranks"] and info["iterations"] == ref["iterations"]
    else:
        y, info, ref = followed_parity(ctx, [a, b], "mul", p["tol"], p["max_rank"], gpu_kw=dict(overlap=overlap),
                                       points=pts, gpu=gpu)
        _followed[key] = ref
    rep = ref["follow"]
    assert rep["updates"] == 39 * (1 + 2 * info["iterations"])
    print(f"\nchi={chi} overlap={overlap}: {rep['updates']} updates, {rep['pivots']} pivots checked, "
          f"{rep['differ']} near-tie choices differ from the oracle's own argmax; "
          f"iterations {info['iterations']}, max rank {max(info['ranks'])}")
    # the output against the exact product on the same points (error control of Sec. 2.6)
    exact = tt_eval(a, pts) * tt_eval(b, pts)
    err = np.abs(tt_eval(y, pts) - exact).max() / np.abs(exact).max()
    assert err <= 20 * info["max_eps"] / info["scale"] + 1e-12


def _random_cores(rng, dims, rank, cplx):
    ranks = [1] + [rank] * (len(dims) - 1) + [1]
    cores = []
    for s, d in enumerate(dims):
        c = rng.uniform(-1, 1, (ranks[s], d, ranks[s + 1]))
        if cplx:
            c = c + 1j * rng.uniform(-1, 1, c.shape)
        cores.append(c)
    return cores


@pytest.mark.parametrize("dims,rank,max_rank,cplx,variant", [
    ((600, 400), 5, 400, False, "cluster kernel: 600 x 400 real"),
    ((8, 8, 8, 8), 7, 40, True, "cluster kernel: 8 x 320 complex (bond 0)"),
    ((700, 700), 5, 700, False, "grid kernel: 700 x 700 real"),
    ((8, 8, 8, 8, 8, 8), 5, 64, True, "grid kernel: 512 x 512 complex (bond 2)"),
])
def test_whole_call_through_each_pivot_variant(ctx, dims, rank, max_rank, cplx, variant):
    rng = np.random.default_rng(sum(dims) + rank)
    a = _random_cores(rng, dims, rank, cplx)
    b = _random_cores(rng, dims, rank, cplx)
    npts = int(np.prod(dims, dtype=np.float64)) if np.prod(dims, dtype=np.float64) <= 2 ** 20 else None
    pts = None
    if npts is None:
        pts = np.stack([rng.integers(0, d, 20000) for d in dims], axis=1)
    y, info, ref = followed_parity(ctx, [a, b], "mul", 1e-12, max_rank, points=pts)
    assert max(info["ranks"]) == min(rank * rank, max_rank)  # the product's exact rank, or the cap
    if pts is None and rank * rank <= max_rank:
        exact = tt_full(a) * tt_full(b)
        assert np.abs(tt_full(y) - exact).max() <= 1e-10 * np.abs(exact).max()
