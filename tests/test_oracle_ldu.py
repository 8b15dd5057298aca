"""Pins for the oracle's Algorithm 2 (LDU / prrLU) and Algorithm 3 (CI).

References that are not the oracle itself:
  * an independent complete-pivoting LU written with masks and explicit rank-1 sums
    (no swaps, no in-place storage) - the textbook definition of Gaussian elimination
    with complete pivoting (Golub & Van Loan, Sec. 3.4.8);
  * brute-force identities: M - L D U vanishes on the pivot rows and columns (cross
    interpolation, Sec. 2.7) and equals the Schur complement, so in full search its
    largest entry is the error estimate (reading R2).
"""

import numpy as np
import pytest

from oracle import ldu, crossinterpolate, magnitude


def complete_pivot_reference(M, kmax, tau):
    """Masked Gaussian elimination with complete pivoting (independent restatement)."""
    R = np.array(M, dtype=M.dtype, copy=True)
    m, n = R.shape
    rows_used = np.zeros(m, bool)
    cols_used = np.zeros(n, bool)
    piv = []
    while len(piv) < min(m, n):
        best, bi, bj, bkey = None, -1, -1, -1.0
        for i in range(m):
            if rows_used[i]:
                continue
            for j in range(n):
                if cols_used[j]:
                    continue
                v = R[i, j]
                key = (v.real * v.real + v.imag * v.imag) if np.iscomplexobj(R) else abs(v)
                if key > bkey:  # strict: first (lowest linear index) wins ties
                    bkey, bi, bj, best = key, i, j, v
        mag = abs(best)
        if len(piv) == kmax or (len(piv) >= 1 and mag <= tau):
            break
        piv.append((bi, bj, best))
        col = R[:, bj].copy()
        row = R[bi, :].copy()
        if best != 0:
            for i in range(m):
                for j in range(n):
                    if not rows_used[i] and not cols_used[j]:
                        R[i, j] = R[i, j] - col[i] * row[j] / best
        rows_used[bi] = True
        cols_used[bj] = True
    return piv, R, rows_used, cols_used


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("cplx", [False, True])
def test_ldu_matches_complete_pivoting(seed, cplx):
    rng = np.random.default_rng(seed)
    m, n = rng.integers(1, 13, size=2)
    M = rng.standard_normal((m, n))
    if cplx:
        M = M + 1j * rng.standard_normal((m, n))
    f = ldu(M, 0.0, min(m, n))
    piv, _, _, _ = complete_pivot_reference(M, min(m, n), 0.0)
    assert f["k"] == len(piv) == min(m, n)
    assert list(f["I"]) == [p[0] for p in piv]
    assert list(f["J"]) == [p[1] for p in piv]
    np.testing.assert_allclose(f["D"], [p[2] for p in piv], rtol=1e-11, atol=1e-12)
    # full rank: exact factorisation
    rec = f["L"] @ (f["D"][:, None] * f["U"])
    assert np.abs(rec - M).max() <= 1e-12 * max(1.0, np.abs(M).max())
    # unit triangular in pivot order, bounded by 1 (complete pivoting)
    LI = f["L"][f["I"], :]
    UJ = f["U"][:, f["J"]]
    np.testing.assert_allclose(np.diag(LI), 1.0)
    np.testing.assert_allclose(np.diag(UJ), 1.0)
    assert np.abs(np.triu(LI, 1)).max(initial=0) == 0.0
    assert np.abs(np.tril(UJ, -1)).max(initial=0) == 0.0
    assert magnitude(f["L"]).max() <= 1 + 1e-12 and magnitude(f["U"]).max() <= 1 + 1e-12


@pytest.mark.parametrize("seed", range(8))
def test_truncated_residual_is_schur_block(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = rng.integers(4, 15, size=2)
    M = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-3, 3, size=(m, 1))
    kmax = int(rng.integers(1, min(m, n)))
    f = ldu(M, 0.0, kmax)
    piv, R, ru, cu = complete_pivot_reference(M, kmax, 0.0)
    assert f["k"] == kmax == len(piv)
    resid = M - f["L"] @ (f["D"][:, None] * f["U"])
    scale = np.abs(M).max()
    # cross interpolation: exact on pivot rows and columns
    assert np.abs(resid[f["I"], :]).max() <= 1e-12 * scale
    assert np.abs(resid[:, f["J"]]).max() <= 1e-12 * scale
    # residual equals the independent Schur complement, and eps is its max
    np.testing.assert_allclose(resid[np.ix_(~ru, ~cu)], R[np.ix_(~ru, ~cu)], atol=1e-11 * scale)
    assert abs(f["eps"] - np.abs(resid).max()) <= 1e-11 * scale


def test_tolerance_stop_and_rank():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((9, 3))
    B = rng.standard_normal((3, 11))
    M = A @ B  # exact rank 3
    f = ldu(M, 1e-10 * np.abs(M).max(), 100)
    assert f["k"] == 3
    assert f["eps"] <= 1e-10 * np.abs(M).max()
    g = crossinterpolate(M, 1e-10 * np.abs(M).max(), 100, "left")
    assert np.abs(g["A"] @ g["B"] - M).max() <= 1e-12 * np.abs(M).max()
    D = np.diag([5.0, -3.0, 1e-12, 2e-13])
    f = ldu(D, 1e-10, 10)
    assert f["k"] == 2 and list(f["I"]) == [0, 1] and f["eps"] == 1e-12


def test_degenerate_cases():
    f = ldu(np.zeros((3, 4)), 0.0, 3)
    assert f["k"] == 1 and f["D"][0] == 0 and f["eps"] == 0.0
    assert (f["I"][0], f["J"][0]) == (0, 0)
    f = ldu(np.ones((3, 3)), 1e-14, 3)  # all ties: lowest linear index, then exact rank 1
    assert (f["I"][0], f["J"][0]) == (0, 0) and f["k"] == 1 and f["eps"] == 0.0
    M = np.zeros((3, 4))
    M[2, 0] = -2.0
    M[0, 3] = 2.0  # equal magnitudes: (0, 3) has linear index 3 < 8
    f = ldu(M, 0.0, 1)
    assert (f["I"][0], f["J"][0]) == (0, 3) and f["eps"] == 2.0
    f = ldu(np.array([[3.0]]), 0.0, 5)
    assert f["k"] == 1 and f["eps"] == 0.0


@pytest.mark.parametrize("side", ["left", "right"])
@pytest.mark.parametrize("cplx", [False, True])
def test_crossinterpolate_factors(side, cplx):
    rng = np.random.default_rng(3)
    M = rng.standard_normal((10, 7))
    if cplx:
        M = M + 1j * rng.standard_normal((10, 7))
    g = crossinterpolate(M, 0.0, 4, side)
    I, J = g["I"], g["J"]
    AB = g["A"] @ g["B"]
    scale = np.abs(M).max()
    assert np.abs(AB[I, :] - M[I, :]).max() <= 1e-12 * scale
    assert np.abs(AB[:, J] - M[:, J]).max() <= 1e-12 * scale
    if side == "left":
        np.testing.assert_allclose(g["A"][I, :], np.eye(4), atol=1e-12)
        np.testing.assert_allclose(g["B"], M[I, :], atol=1e-12 * scale)
    else:
        np.testing.assert_allclose(g["B"][:, J], np.eye(4), atol=1e-12)
        np.testing.assert_allclose(g["A"], M[:, J], atol=1e-12 * scale)
