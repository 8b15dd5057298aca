"""The allocation-free pivot search (aci_k_prrlu_static) against the oracle and the regular entry.

aci_k_prrlu_static serves callers that may not allocate device memory (a host application that
owns all device memory, a fixed memory budget, code that must not enter an allocator): it runs
the same pivot search with its scratch in a file-scope device array. These tests call it through
the C ABI several times in a row, on matrices at the corners of its documented limits (4096 x 64
and 64 x 4096 real, 512 x 512 complex, 4096 x 64 complex) and on blocks that take each pivot-search
variant (the 16-CTA register kernel, the shared-memory cluster kernel, the cooperative grid
kernel), and check each result against the oracle's Algorithm 2 (tests/test_gpu_kernels.py's
comparison, pivots exact up to the first near-tie) and against aci_k_prrlu on the same input. A
second pair of calls checks that the calls allocate nothing: torch's allocator counters and the
device's free memory are unchanged across them. The file is collected last so that a
stop-at-first-failure run has run every other test first.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
from tests.test_gpu_kernels import _compare_prrlu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_00037_gb300 import binding
    lib = binding.load_library()
    ctx = binding.Context(0)
    yield lib, ctx, binding
    ctx.close()


def _static_prrlu(lib, binding, M, tau, chimax, outs=None):
    m, n = M.shape
    kc = min(m, n, chimax)
    if outs is None:
        outs = (torch.empty(kc, dtype=torch.int32, device=M.device), torch.empty(kc, dtype=torch.int32, device=M.device),
                torch.empty(kc, dtype=M.dtype, device=M.device), torch.zeros((kc, m), dtype=M.dtype, device=M.device),
                torch.zeros((kc, n), dtype=M.dtype, device=M.device))
    pr, pc, D, Lm, Um = outs
    k = C.c_int32()
    eps = C.c_double()
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.aci_k_prrlu_static(C.c_void_p(stream), binding._dtype_code(M), M.data_ptr(), m, n, float(tau),
                                int(chimax), pr.data_ptr(), pc.data_ptr(), D.data_ptr(), Lm.data_ptr(),
                                Um.data_ptr(), C.byref(k), C.byref(eps))
    assert st == 0, binding.STATUS.get(st, st)
    kk = k.value
    return dict(I=pr[:kk].cpu().numpy(), J=pc[:kk].cpu().numpy(), D=D[:kk].cpu().numpy(), k=kk,
                eps=eps.value, L=Lm[:kk].T.cpu().numpy(), U=Um[:kk].cpu().numpy())


def _matrix(seed, m, n, cplx, rank=None):
    rng = np.random.default_rng(seed)
    r = min(m, n) if rank is None else rank
    U = rng.standard_normal((m, r))
    V = rng.standard_normal((r, n))
    if cplx:
        U = U + 1j * rng.standard_normal(U.shape)
        V = V + 1j * rng.standard_normal(V.shape)
    return (U * (10.0 ** -np.linspace(0, 10, r))) @ V


CASES = [  # (m, n, complex, taurel, chimax): in call order
    (300, 200, False, 0.0, 150),     # register kernel
    (64, 96, True, 1e-8, 40),        # register kernel, complex
    (300, 300, True, 1e-8, 120),     # complex, 4 m n > 2^18: the cooperative grid kernel
    (4096, 64, False, 1e-10, 64),    # corner m = 4096 real: cluster kernel, block in shared memory
    (64, 4096, False, 1e-10, 64),    # corner n = 4096 real
    (512, 512, True, 1e-10, 96),     # corner m n = 2^18 complex: grid kernel, grid capped by the array
    (4096, 64, True, 1e-10, 64),     # corner m = 4096 complex: grid kernel, grid capped by the array
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_static_prrlu_matches_oracle_and_regular_entry(env, case):
    lib, ctx, binding = env
    m, n, cplx, taurel, chimax = CASES[case]
    M = _matrix(100 + case, m, n, cplx, rank=min(m, n, 160))
    Md = torch.from_numpy(M).cuda()
    tau = taurel * np.abs(M).max()
    got = _static_prrlu(lib, binding, Md, tau, chimax)
    _compare_prrlu(got, oracle.ldu(M, tau, chimax), M)
    ref = ctx.prrlu(Md, tau, chimax)
    assert got["k"] == ref["k"]
    assert list(got["I"]) == list(ref["I"]) and list(got["J"]) == list(ref["J"])
    assert np.array_equal(got["D"], ref["D"])


def test_static_prrlu_two_calls_in_a_row_allocate_nothing(env):
    lib, ctx, binding = env
    M1 = torch.from_numpy(_matrix(1, 300, 300, True)).cuda()
    M2 = torch.from_numpy(_matrix(2, 64, 96, False)).cuda()
    tau2 = 1e-9 * float(M2.abs().max())
    o1 = (torch.empty(96, dtype=torch.int32, device="cuda"), torch.empty(96, dtype=torch.int32, device="cuda"),
          torch.empty(96, dtype=torch.complex128, device="cuda"),
          torch.zeros((96, 300), dtype=torch.complex128, device="cuda"),
          torch.zeros((96, 300), dtype=torch.complex128, device="cuda"))
    o2 = (torch.empty(40, dtype=torch.int32, device="cuda"), torch.empty(40, dtype=torch.int32, device="cuda"),
          torch.empty(40, dtype=torch.float64, device="cuda"), torch.zeros((40, 64), dtype=torch.float64, device="cuda"),
          torch.zeros((40, 96), dtype=torch.float64, device="cuda"))
    # warm-up of both shapes: the first call sets up the array's address, and each kernel's first
    # launch may load its module
    _static_prrlu(lib, binding, M1, 0.0, 96, o1)
    _static_prrlu(lib, binding, M2, tau2, 40, o2)
    torch.cuda.synchronize()
    before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    free0, _ = torch.cuda.mem_get_info()
    a = _static_prrlu(lib, binding, M1, 0.0, 96, o1)
    b = _static_prrlu(lib, binding, M2, tau2, 40, o2)
    torch.cuda.synchronize()
    after = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    free1, _ = torch.cuda.mem_get_info()
    assert after == before  # no device allocation through torch's allocator
    assert free1 == free0   # nor any other device allocation
    r1 = ctx.prrlu(M1, 0.0, 96)
    r2 = ctx.prrlu(M2, tau2, 40)
    assert list(a["I"]) == list(r1["I"]) and list(a["J"]) == list(r1["J"])
    assert list(b["I"]) == list(r2["I"]) and list(b["J"]) == list(r2["J"])
    np.testing.assert_array_equal(b["D"], r2["D"])


def test_static_prrlu_rejects_sizes_beyond_its_array(env):
    lib, ctx, binding = env
    M = torch.zeros((600, 600), dtype=torch.float64, device="cuda")  # 360000 > 262144 entries
    pr = torch.empty(10, dtype=torch.int32, device="cuda")
    D = torch.empty(10, dtype=torch.float64, device="cuda")
    k, eps = C.c_int32(), C.c_double()
    st = lib.aci_k_prrlu_static(None, 0, M.data_ptr(), 600, 600, 0.0, 10, pr.data_ptr(), pr.data_ptr(),
                                D.data_ptr(), None, None, C.byref(k), C.byref(eps))
    assert st == -2  # ACI_E_SHAPE
