"""Failure detection without a GPU fault.

Every device-side wait of the library is bounded: the pivot search's waits on other CTAs'
exchange words (cooperative grid variant) and on its pushed pivot row and column (2D register
variant), and the tensor-core contraction's waits on its copy and multiply pipeline. aci_set_wait_limits shrinks those bounds to a few polls, so that an ordinary
call runs them out: the kernels record a timeout, let their copies in flight finish, return, and
the call reports ACI_E_TIMEOUT; restoring the defaults, the same context computes the right
result again. An allocator hook that returns NULL makes a call fail with ACI_E_ALLOC and leave
its output untouched. Nothing here traps, faults or hangs a GPU."""

import ctypes as C

import numpy as np
import pytest

import oracle
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
    c.set_wait_limits(0, 0)
    c.close()


def _graded(seed, m, n, cplx=False):
    rng = np.random.default_rng(seed)
    r = min(m, n)
    U, V = rng.standard_normal((m, r)), rng.standard_normal((r, n))
    if cplx:
        U, V = U + 1j * rng.standard_normal(U.shape), V + 1j * rng.standard_normal(V.shape)
    return (U * 10.0 ** -np.linspace(0, 12, r)) @ V


def test_pivot_search_exchange_wait_runs_out(ctx):
    from paper_2604_00037_gb300.binding import AciError
    M = _graded(1, 700, 700)  # 700 x 700 real: the cooperative grid variant
    Md = torch.from_numpy(M).cuda()
    tau = 1e-10 * np.abs(M).max()
    ctx.set_wait_limits(exchange_polls=1)
    try:
        with pytest.raises(AciError, match="ACI_E_TIMEOUT"):
            ctx.prrlu(Md, tau, 300)
    finally:
        ctx.set_wait_limits(0, 0)
    _compare_prrlu(ctx.prrlu(Md, tau, 300), oracle.ldu(M, tau, 300), M)  # the context is usable


def test_pivot_search_push_wait_runs_out(ctx):
    """1000 x 200 real: the 2D register variant (an 8 x 2 grid of CTAs), whose threads wait on the
    mbarrier that the pushed pivot row and column entries complete; one non-blocking test per wait
    runs out, and a run-out wait stops every CTA at the next exchange."""
    from paper_2604_00037_gb300.binding import AciError
    M = _graded(4, 1000, 200)
    Md = torch.from_numpy(M).cuda()
    tau = 1e-10 * np.abs(M).max()
    ctx.set_wait_limits(exchange_polls=1)
    try:
        with pytest.raises(AciError, match="ACI_E_TIMEOUT"):
            ctx.prrlu(Md, tau, 150)
    finally:
        ctx.set_wait_limits(0, 0)
    _compare_prrlu(ctx.prrlu(Md, tau, 150), oracle.ldu(M, tau, 150), M)  # the context is usable


def test_tensor_core_pipeline_wait_runs_out(ctx):
    from paper_2604_00037_gb300.binding import AciError
    rng = np.random.default_rng(2)
    A = torch.from_numpy(rng.standard_normal((1024, 512)) + 1j * rng.standard_normal((1024, 512))).cuda()
    B = torch.from_numpy(rng.standard_normal((512, 768)) + 1j * rng.standard_normal((512, 768))).cuda()
    ctx.set_wait_limits(pipeline_polls=1)
    try:
        with pytest.raises(AciError, match="ACI_E_TIMEOUT"):
            ctx.pi_block([A], [B], "abs2_mul", precision="bf16x6")
    finally:
        ctx.set_wait_limits(0, 0)
    Pi, mx = ctx.pi_block([A], [B], "abs2_mul", precision="bf16x6")
    ref = (A @ B).cpu().numpy()
    ref = (ref.real ** 2 + ref.imag ** 2) * ref
    assert np.abs(Pi.cpu().numpy() - ref).max() <= 1e-7 * np.abs(ref).max()


def test_whole_call_reports_the_timeout(ctx):
    from paper_2604_00037_gb300.binding import AciError
    rng = np.random.default_rng(3)
    a = [rng.uniform(-1, 1, (1, 700, 5)), rng.uniform(-1, 1, (5, 700, 1))]
    b = [rng.uniform(-1, 1, (1, 700, 5)), rng.uniform(-1, 1, (5, 700, 1))]
    dev = lambda tt: [torch.from_numpy(c).cuda() for c in tt]
    ctx.set_wait_limits(exchange_polls=1)
    try:
        with pytest.raises(AciError, match="ACI_E_TIMEOUT"):
            ctx.elementwise(dev(a), dev(b), "mul", 1e-12, 700)
    finally:
        ctx.set_wait_limits(0, 0)
    y, info = ctx.elementwise(dev(a), dev(b), "mul", 1e-12, 700)
    assert max(info["ranks"]) == 25


def test_null_allocator_gives_alloc_error_and_leaves_the_output():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_00037_gb300 import binding
    lib = binding.load_library()
    calls = []

    def alloc(nbytes, user):
        calls.append(nbytes)
        return None  # the allocator refuses every request

    def free(ptr, user):
        pass

    afn, ffn = binding.ALLOC_FN(alloc), binding.FREE_FN(free)
    h = C.c_void_p()
    assert lib.aci_create(C.byref(h), 0, None, afn, ffn, None) == 0
    try:
        rng = np.random.default_rng(4)
        cores = [torch.from_numpy(rng.uniform(-1, 1, s)).cuda() for s in ((1, 2, 3), (3, 2, 3), (3, 2, 1))]
        A = binding._TTArg(cores)
        out = binding.AciTT()
        st = lib.aci_elementwise(h, C.byref(A.tt), C.byref(A.tt), binding.make_op("mul"), 1e-10, 16, C.byref(out))
        assert st == -4  # ACI_E_ALLOC
        assert calls, "the hook was asked"
        assert "allocation" in lib.aci_last_error(h).decode()
        assert out.L == 0 and not out.core and not out.rank  # untouched
    finally:
        lib.aci_destroy(h)
