"""Pins for the oracle's rook-search prrLU (reading R11 in oracle/algorithms.py).

References that are not the oracle itself:
  * the Schur complement after pivots (I_p, J_p) written with the cross formula
    R_p = M - M[:, J_p] M[I_p, J_p]^-1 M[I_p, :] (Sec. 2.7), solved with numpy, which the
    oracle never uses (it forms residuals from its own L, D, U);
  * what any rook pivot must satisfy: it is the largest residual entry of its column over the
    unused rows, and it is the largest of its row too when the search stopped at a fixed point;
  * cross interpolation: M - L D U vanishes on the pivot rows and columns, and on a matrix of
    exact rank r the factorisation is exact after r pivots;
  * the first pivot is the global maximum (the search starts from its column).
"""

import numpy as np
import pytest

from oracle import ldu_rook, ldu, magnitude, aci, pivot_key
from synthetic.tt import tt_full, tt_random_uniform


def key(v):
    return (v.real * v.real + v.imag * v.imag) if np.iscomplexobj(v) else np.abs(v)


def schur(M, I, J):
    """Residual after eliminating rows I and columns J (cross formula), zero on them."""
    if len(I) == 0:
        return M.copy()
    P = M[np.ix_(I, J)]
    R = M - M[:, J] @ np.linalg.solve(P, M[I, :])
    R[I, :] = 0
    R[:, J] = 0
    return R


def rand(rng, m, n, cplx):
    M = rng.standard_normal((m, n))
    if cplx:
        M = M + 1j * rng.standard_normal((m, n))
    return M


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("cplx", [False, True])
def test_rook_pivots_are_column_maxima_of_the_schur_complement(seed, cplx):
    rng = np.random.default_rng(seed)
    m, n = (int(x) for x in rng.integers(2, 14, size=2))
    M = rand(rng, m, n, cplx)
    f = ldu_rook(M, 0.0, 64)
    I, J, D = list(f["I"]), list(f["J"]), f["D"]
    assert f["k"] == min(m, n)
    scale = np.abs(M).max()
    row_max_hits = 0
    for p in range(f["k"]):
        R = schur(M, I[:p], J[:p])
        r, c = I[p], J[p]
        assert abs(D[p] - R[r, c]) <= 1e-10 * scale * (1 + p)
        free_r = np.ones(m, bool)
        free_r[I[:p]] = False
        free_c = np.ones(n, bool)
        free_c[J[:p]] = False
        colkeys = key(R[:, c])[free_r]
        assert key(R[r, c]) >= colkeys.max() * (1 - 1e-9)
        row_max_hits += key(R[r, c]) >= key(R[r, :])[free_c].max() * (1 - 1e-9)
    # a fixed point makes the pivot a row maximum too; the fourth-hop exit is the exception
    assert row_max_hits >= f["k"] // 2


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("cplx", [False, True])
def test_rook_factors_interpolate_the_pivot_cross(seed, cplx):
    rng = np.random.default_rng(100 + seed)
    m, n = 11, 9
    M = rand(rng, m, n, cplx)
    f = ldu_rook(M, 0.0, 5)
    A = f["L"] @ (f["D"][:, None] * f["U"])
    I, J = f["I"], f["J"]
    assert np.abs(A[I, :] - M[I, :]).max() <= 1e-12 * np.abs(M).max()
    assert np.abs(A[:, J] - M[:, J]).max() <= 1e-12 * np.abs(M).max()
    # unit triangular in pivot order, zero on rows/columns pivoted earlier
    LI, UJ = f["L"][I, :], f["U"][:, J]
    assert np.allclose(np.diag(LI), 1) and np.allclose(np.triu(LI, 1), 0)
    assert np.allclose(np.diag(UJ), 1) and np.allclose(np.tril(UJ, -1), 0)
    # the residual outside the cross is the Schur complement
    R = schur(M, list(I), list(J))
    assert np.abs((M - A) - R).max() <= 1e-10 * np.abs(M).max()
    # epsilon is the magnitude of the next rook pivot: an entry of R, at most its maximum
    assert f["eps"] <= magnitude(R).max() * (1 + 1e-12)
    assert np.any(np.isclose(magnitude(R), f["eps"], rtol=1e-9, atol=0))


@pytest.mark.parametrize("rank", [1, 3, 6])
@pytest.mark.parametrize("cplx", [False, True])
def test_rook_is_exact_on_low_rank(rank, cplx):
    rng = np.random.default_rng(rank)
    m, n = 14, 12
    M = rand(rng, m, rank, cplx) @ rand(rng, rank, n, cplx)
    f = ldu_rook(M, 1e-10 * np.abs(M).max(), 64)
    assert f["k"] == rank
    A = f["L"] @ (f["D"][:, None] * f["U"])
    assert np.abs(A - M).max() <= 1e-10 * np.abs(M).max()
    assert f["eps"] <= 1e-10 * np.abs(M).max()


def test_rook_first_pivot_is_global_max_and_ties_go_low():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((7, 9))
    f = ldu_rook(M, 0.0, 3)
    i, j = np.unravel_index(np.argmax(np.abs(M)), M.shape)
    assert (f["I"][0], f["J"][0]) == (i, j)
    E = np.ones((4, 5))
    g = ldu_rook(E, 1e-12, 4)
    assert g["k"] == 1 and (g["I"][0], g["J"][0]) == (0, 0) and g["eps"] == 0.0


def test_rook_equals_full_search_when_the_maximum_is_a_rook_point():
    """A rank-one matrix x y^T: the global maximum is the largest of its row and column, so both
    searches take the same single pivot and stop with the same (zero) estimate."""
    x = np.array([0.3, -2.0, 1.1, 0.7])
    y = np.array([1.5, -0.2, 0.9, -3.0, 0.4])
    M = np.outer(x, y)
    fr, ff = ldu_rook(M, 1e-13, 4), ldu(M, 1e-13, 4)
    assert fr["k"] == ff["k"] == 1
    assert (fr["I"][0], fr["J"][0]) == (ff["I"][0], ff["J"][0])
    assert fr["D"][0] == ff["D"][0]


def test_rook_degenerate_shapes():
    Z = np.zeros((3, 4))
    f = ldu_rook(Z, 0.0, 4)
    assert f["k"] == 1 and f["D"][0] == 0 and f["eps"] == 0.0
    assert f["L"][f["I"][0], 0] == 1 and f["U"][0, f["J"][0]] == 1
    one = ldu_rook(np.array([[2.5]]), 0.0, 4)
    assert one["k"] == 1 and one["D"][0] == 2.5 and one["eps"] == 0.0
    col = np.array([[1.0], [-4.0], [2.0]])
    g = ldu_rook(col, 0.0, 4)
    assert g["k"] == 1 and g["I"][0] == 1 and g["eps"] == 0.0
    row = col.T
    h = ldu_rook(row, 0.0, 4)
    assert h["k"] == 1 and h["J"][0] == 1


def test_aci_rook_mode_matches_dense_product():
    """The whole method with rook pivots reproduces f on a full grid to its tolerance."""
    rng = np.random.default_rng(11)
    a = tt_random_uniform(rng, 6, 2, 3, low=-1, high=1)
    b = tt_random_uniform(rng, 6, 2, 4, low=-1, high=1)
    out = aci([a, b], "mul", 1e-12, 64, pivot_mode="rook")
    exact = tt_full(a) * tt_full(b)
    assert np.abs(tt_full(out["Y"]) - exact).max() <= 1e-10 * np.abs(exact).max()
    c = tt_random_uniform(rng, 5, 3, 3, dtype=np.complex128, low=-1, high=1)
    out = aci([c], "abs2_mul", 1e-12, 200, pivot_mode="rook")
    C = tt_full(c)
    exact = np.abs(C) ** 2 * C
    assert np.abs(tt_full(out["Y"]) - exact).max() <= 1e-9 * np.abs(exact).max()
