"""The allocation-free pivot search (aci_k_prrlu_static) against the regular entry point.

aci_k_prrlu_static serves callers that may not allocate device memory (a host application that
owns all device memory, a fixed memory budget, code that must not enter an allocator): it runs
the same pivot search with its scratch in a file-scope device array. This test calls it through
the C ABI twice in a row, on two different matrices, and checks each result against
aci_k_prrlu on the same input, with the tolerances of the other pivot-search tests. It lives in
a file collected last so that a stop-at-first-failure run has run every other test first.
"""

import ctypes as C

import numpy as np
import pytest

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


def _static_prrlu(lib, binding, M, tau, chimax):
    m, n = M.shape
    kc = min(m, n, chimax)
    pr = torch.empty(kc, dtype=torch.int32, device=M.device)
    pc = torch.empty(kc, dtype=torch.int32, device=M.device)
    D = torch.empty(kc, dtype=M.dtype, device=M.device)
    Lm = torch.zeros((kc, m), dtype=M.dtype, device=M.device)
    Um = torch.zeros((kc, n), dtype=M.dtype, device=M.device)
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


def _matrix(seed, m, n, cplx):
    rng = np.random.default_rng(seed)
    r = min(m, n)
    U = rng.standard_normal((m, r))
    V = rng.standard_normal((r, n))
    if cplx:
        U = U + 1j * rng.standard_normal(U.shape)
        V = V + 1j * rng.standard_normal(V.shape)
    return (U * (10.0 ** -np.linspace(0, 10, r))) @ V


def _same(got, ref, scale):
    assert got["k"] == ref["k"]
    assert list(got["I"]) == list(ref["I"]) and list(got["J"]) == list(ref["J"])
    assert abs(got["eps"] - ref["eps"]) <= 1e-12 * scale
    np.testing.assert_allclose(got["D"], ref["D"], atol=1e-12 * scale, rtol=1e-12)
    bound = 1e-13 * scale / np.abs(ref["D"]) + 1e-12
    assert (np.abs(got["L"] - ref["L"]) <= bound[None, :]).all()
    assert (np.abs(got["U"] - ref["U"]) <= bound[:, None]).all()


def test_static_prrlu_matches_regular_entry_two_calls_in_a_row(env):
    lib, ctx, binding = env
    cases = [(_matrix(1, 300, 200, False), 0.0, 150),     # first call: real, larger
             (_matrix(2, 64, 96, True), 1e-8, 40)]         # second call: complex, smaller
    for M, taurel, chimax in cases:
        Md = torch.from_numpy(M).cuda()
        scale = np.abs(M).max()
        tau = taurel * scale
        got = _static_prrlu(lib, binding, Md, tau, chimax)
        ref = ctx.prrlu(Md, tau, chimax)
        _same(got, ref, scale)


def test_static_prrlu_rejects_sizes_beyond_its_array(env):
    lib, ctx, binding = env
    M = torch.zeros((600, 600), dtype=torch.float64, device="cuda")  # 360000 > 262144 entries
    pr = torch.empty(10, dtype=torch.int32, device="cuda")
    D = torch.empty(10, dtype=torch.float64, device="cuda")
    k, eps = C.c_int32(), C.c_double()
    st = lib.aci_k_prrlu_static(None, 0, M.data_ptr(), 600, 600, 0.0, 10, pr.data_ptr(), pr.data_ptr(),
                                D.data_ptr(), None, None, C.byref(k), C.byref(eps))
    assert st == -2  # ACI_E_SHAPE
