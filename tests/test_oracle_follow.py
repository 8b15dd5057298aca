"""The oracle's follow mode (oracle.ldu / oracle.aci with ``follow=``), which the GPU parity tests
use to check every pivot of full-size runs. Reading R4: where two candidates of Algorithm 2's
argmax differ by less than the rounding of the Schur entries, either choice is correct; the
follow mode takes the other implementation's choice there and flags every choice that is not
within the slack of the maximum, and every rank that stops or continues against the stop test.

Pins: following its own history reproduces a plain run bit for bit; an exact tie may be broken
either way (counted in ``differ``, no breach); a reversed pivot order, a pivot below the maximum,
a rank that stops early and a rank that runs past the stop test are each flagged."""

import numpy as np

import oracle
from synthetic import config_inputs, tt_full, tt_random_uniform


def test_following_own_history_reproduces_the_plain_run():
    p = config_inputs(1)
    a, b = p["inputs"]
    r = oracle.aci([a, b], "mul", p["tol"], p["max_rank"])
    f = oracle.aci([a, b], "mul", p["tol"], p["max_rank"], follow=r["history"])
    rep = f["follow"]
    assert rep["violations"] == [] and rep["differ"] == 0
    assert rep["updates"] == len(r["history"]) == 11 * (1 + 2 * r["iterations"])
    assert f["ranks"] == r["ranks"] and f["iterations"] == r["iterations"]
    assert all(np.array_equal(x, y) for x, y in zip(f["Y"], r["Y"]))


def test_exact_tie_may_go_either_way():
    M = np.array([[1.0, 0.2], [0.3, -1.0]])  # |M00| == |M11|: R4 picks (0, 0), (1, 1) is as large
    own = oracle.ldu(M, 0.0, 2)
    assert (own["I"][0], own["J"][0]) == (0, 0)
    f = oracle.ldu(M, 0.0, 2, follow=([1, 0], [1, 0]), slack=1e-15)
    assert f["violations"] == [] and f["differ"] == 1
    assert (f["I"][0], f["J"][0]) == (1, 1)
    assert np.allclose(f["L"] @ np.diag(f["D"]) @ f["U"], M)


def test_breaches_are_flagged():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((9, 7))
    own = oracle.ldu(M, 1e-3, 7)
    I, J = list(own["I"]), list(own["J"])
    rev = oracle.ldu(M, 1e-3, 7, follow=(I[::-1], J[::-1]), slack=1e-12)
    assert rev["violations"] and "below the maximum" in rev["violations"][0][1]
    early = oracle.ldu(M, 1e-3, 7, follow=(I[:3], J[:3]), slack=1e-12)
    assert any("stops early" in v[1] for v in early["violations"])
    # one extra pivot beyond the rank cap
    capped = oracle.ldu(M, 0.0, 3)
    over = oracle.ldu(M, 0.0, 3, follow=(list(capped["I"]) + [8], list(capped["J"]) + [6]), slack=1e-12)
    assert any("continues past" in v[1] for v in over["violations"])
    # a pivot in a row that is already used
    used = oracle.ldu(M, 1e-3, 7, follow=([I[0], I[0]] + I[2:], J), slack=1e-12)
    assert any("used row" in v[1] for v in used["violations"])


def test_a_perturbed_history_is_caught_in_a_whole_call():
    rng = np.random.default_rng(11)
    a = tt_random_uniform(rng, 6, 2, 3, low=-1, high=1)
    b = tt_random_uniform(rng, 6, 2, 3, low=-1, high=1)
    r = oracle.aci([a, b], "mul", 1e-12, 32)
    h = dict(r["history"])
    key = (2, 2)  # right-to-left update of the first iteration at bond 2
    rows, cols = h[key]
    h[key] = (rows[::-1].copy(), cols[::-1].copy())
    f = oracle.aci([a, b], "mul", 1e-12, 32, follow=h)
    assert any(v[:2] == key for v in f["follow"]["violations"])
    # the unperturbed history reproduces the exact product
    g = oracle.aci([a, b], "mul", 1e-12, 32, follow=r["history"])
    assert g["follow"]["violations"] == []
    exact = tt_full(a) * tt_full(b)
    assert np.abs(tt_full(g["Y"]) - exact).max() <= 1e-12 * np.abs(exact).max()
