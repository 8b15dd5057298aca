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
