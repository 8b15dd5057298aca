"""Planted mistakes in the oracle must fail a pin (the pins are sensitive, not vacuous).

Each case patches one plausible mistake into a copy of the oracle's Algorithm 2 on the
CPU (wrong Schur sign, dropped column swap, pivot by value instead of magnitude) and
checks that the brute-force references used by the pin tests reject it.
"""

import numpy as np
import pytest

import oracle.algorithms as oa
from synthetic import tt_full, config_inputs


def _mutant_ldu(kind):
    src_ldu = oa.ldu

    def ldu(M, tau, chimax):
        S = np.array(M, copy=True)
        m, n = S.shape
        I, J = np.arange(m), np.arange(n)
        chi = 0
        while chi < min(m, n):
            sub = S[chi:, chi:]
            key = sub.real if kind == "value_not_magnitude" else oa.pivot_key(sub)
            i, j = np.unravel_index(int(np.argmax(key)), key.shape)
            i += chi
            j += chi
            if chi == chimax or (chi >= 1 and abs(S[i, j]) <= tau):
                break
            S[[i, chi], :] = S[[chi, i], :]
            if kind != "no_col_swap":
                S[:, [j, chi]] = S[:, [chi, j]]
                J[[j, chi]] = J[[chi, j]]
            I[[i, chi]] = I[[chi, i]]
            sign = 1.0 if kind == "schur_sign" else -1.0
            l = S[chi + 1:, chi] / S[chi, chi]
            S[chi + 1:, chi + 1:] += sign * np.outer(l, S[chi, chi + 1:])
            chi += 1
        k = chi
        D = np.array([S[p, p] for p in range(k)])
        Lp = np.zeros((m, k))
        Up = np.zeros((k, n))
        for p in range(k):
            Lp[p + 1:, p] = S[p + 1:, p] / D[p]
            Up[p, p + 1:] = S[p, p + 1:] / D[p]
            Lp[p, p] = Up[p, p] = 1
        L = np.zeros_like(Lp)
        U = np.zeros_like(Up)
        L[I, :] = Lp
        U[:, J] = Up
        return dict(L=L, D=D, U=U, I=I[:k].copy(), J=J[:k].copy(), eps=0.0, k=k,
                    best=np.zeros(k), second=np.zeros(k))

    return ldu, src_ldu


def _ldu_pin_fails(mut):
    """The complete-pivoting pin of test_oracle_ldu on a few random matrices."""
    from tests.test_oracle_ldu import complete_pivot_reference
    for seed in range(6):
        rng = np.random.default_rng(seed)
        M = rng.standard_normal((7, 6))
        f = mut(M, 0.0, 6)
        piv, _, _, _ = complete_pivot_reference(M, 6, 0.0)
        if list(f["I"]) != [q[0] for q in piv] or list(f["J"]) != [q[1] for q in piv]:
            return True
        if np.abs(f["L"] @ (f["D"][:, None] * f["U"]) - M).max() > 1e-12 * np.abs(M).max():
            return True
    return False


@pytest.mark.parametrize("kind", ["schur_sign", "no_col_swap", "value_not_magnitude"])
def test_planted_mistake_is_caught(kind, monkeypatch):
    mut, _ = _mutant_ldu(kind)
    if _ldu_pin_fails(mut):
        return
    monkeypatch.setattr(oa, "ldu", mut)
    p = config_inputs(1)
    a, b = p["inputs"]
    try:
        r = oa.aci([a, b], "mul", p["tol"], p["max_rank"], maxiter=4)
        y = tt_full(r["Y"])
        err = np.abs(y - tt_full(a) * tt_full(b)).max() / np.abs(tt_full(a) * tt_full(b)).max()
    except (KeyError, IndexError, ValueError, np.linalg.LinAlgError, FloatingPointError):
        return  # structurally broken: caught
    assert not (err <= 10 * p["tol"]), f"mutant {kind} passed the dense brute-force pin (err={err})"


def _mutant_rook(kind):
    """A copy of the rook search (reading R11) with one planted mistake."""

    def ldu_rook(M, tau, chimax):
        M = np.array(M, copy=True)
        m, n = M.shape
        kcap = min(m, n, chimax)
        L = np.zeros((m, kcap))
        U = np.zeros((kcap, n))
        D = np.zeros(kcap)
        fr = np.ones(m, bool)
        fc = np.ones(n, bool)
        I, J = [], []
        p, c_next = 0, None
        sgn = 1.0 if kind == "resid_sign" else -1.0

        def col_of(c):
            w = U[:p, c] if kind == "missing_D" else D[:p] * U[:p, c]
            return M[:, c] + sgn * (L[:, :p] @ w)

        def row_of(r):
            v = L[r, :p] if kind == "missing_D" else L[r, :p] * D[:p]
            return M[r, :] + sgn * (v @ U[:p, :])

        def amax(v, free):
            return int(np.argmax(np.where(free, np.abs(v), -1.0)))

        while p < min(m, n):
            c0 = int(np.argmax(np.abs(M))) % n if p == 0 else c_next
            col = col_of(c0)
            r1 = amax(col, fr)
            row = row_of(r1)
            c1 = amax(row, fc)
            if c1 == c0:
                r, c = r1, c0
            elif kind == "no_second_hop":
                r, c = r1, c1
            else:
                col = col_of(c1)
                r2 = amax(col, fr)
                r, c = (r1, c1) if r2 == r1 else (r2, c1)
                if r != r1 and kind != "row_from_stale":
                    row = row_of(r)
            piv = col[r]
            if p == chimax or (p >= 1 and abs(piv) <= tau):
                break
            L[:, p] = np.where(fr, col / piv, 0)
            U[p, :] = np.where(fc, row / piv, 0)
            L[r, p] = U[p, c] = 1
            D[p] = piv
            fr[r] = fc[c] = False
            I.append(r)
            J.append(c)
            if fc.any():
                c_next = int(np.argmax(np.where(fc, np.abs(row), -1.0)))
            p += 1
        return dict(L=L[:, :p], D=D[:p], U=U[:p], I=np.array(I), J=np.array(J), eps=0.0, k=p)

    return ldu_rook


def _rook_pin_fails(mut):
    """The Schur-complement and cross-interpolation pins of test_oracle_rook."""
    from tests.test_oracle_rook import schur
    for seed in range(8):
        rng = np.random.default_rng(seed)
        M = rng.standard_normal((8, 7))
        f = mut(M, 0.0, 6)
        I, J = list(f["I"]), list(f["J"])
        if len(set(I)) != len(I) or len(set(J)) != len(J):
            return True
        A = f["L"] @ (f["D"][:, None] * f["U"])
        if np.abs(A[I, :] - M[I, :]).max() > 1e-10 or np.abs(A[:, J] - M[:, J]).max() > 1e-10:
            return True
        for p in range(f["k"]):
            R = schur(M, I[:p], J[:p])
            free = np.ones(8, bool)
            free[I[:p]] = False
            if abs(f["D"][p] - R[I[p], J[p]]) > 1e-9 or abs(R[I[p], J[p]]) < np.abs(R[free, J[p]]).max() * (1 - 1e-9):
                return True
    return False


@pytest.mark.parametrize("kind", ["resid_sign", "missing_D", "no_second_hop", "row_from_stale"])
def test_planted_rook_mistake_is_caught(kind):
    assert _rook_pin_fails(_mutant_rook(kind)), f"rook mutant {kind} passed the pins"


def test_unmutated_rook_copy_passes_the_pins():
    assert not _rook_pin_fails(_mutant_rook("none"))
