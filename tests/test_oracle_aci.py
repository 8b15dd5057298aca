"""Pins for the oracle's Algorithm 1 (ACI) and its assembly of the output (reading R6).

Independent references used here:
  * dense brute force: the elementwise product of the dense inputs on every grid point;
  * exact low-rank products: random TTs with chi_a * chi_b <= chi_hat are reproduced exactly;
  * closed forms: single Fourier modes multiply to one mode (Eq. (quanticsrep) makes every
    mode a rank-1 TT), the Gaussian product of Eq. (gaussians) and the Fourier convolution
    of Eq. (fouriermultiplication);
  * invariants: commutativity, b = 1, real conj, interpolation on the pivot cross (Sec. 2.5),
    nesting of the J sets (Sec. 2.5), and the published SplitMix64 test vector.
"""

import json
import os

import numpy as np
import pytest

import oracle
from oracle.rng import splitmix64
from synthetic import (tt_full, tt_eval, tt_random_uniform, config_inputs, gaussian_pair,
                       fourier_paper_1d)
from synthetic.fields import exp_mode_tt, _site_angles

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rel_err(y, ref):
    return np.abs(y - ref).max() / np.abs(ref).max()


def test_splitmix64_published_vector():
    g = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    out = splitmix64(g["seed"], np.arange(5))
    assert [int(v) for v in out] == [int(s) for s in g["outputs"]]


def test_config1_dense_bruteforce():
    p = config_inputs(1)
    a, b = p["inputs"]
    r = oracle.aci([a, b], "mul", p["tol"], p["max_rank"])
    ref = tt_full(a) * tt_full(b)
    err = rel_err(tt_full(r["Y"]), ref)
    assert err <= 10 * p["tol"], err
    # error estimate is an upper-bound proxy of the dense error (heuristic, reported)
    assert max(r["eps"]) / r["S"] >= 0.1 * err


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("cplx", [False, True])
def test_exact_low_rank_products(seed, cplx):
    rng = np.random.default_rng(seed)
    L = int(rng.integers(3, 10))
    chi = int(rng.integers(1, 5))
    dt = np.complex128 if cplx else np.float64
    a = tt_random_uniform(rng, L, 2, chi, dtype=dt, low=-1, high=1)
    b = tt_random_uniform(rng, L, 2, chi, dtype=dt, low=-1, high=1)
    r = oracle.aci([a, b], "mul", 1e-14, 64, seed=seed)
    assert rel_err(tt_full(r["Y"]), tt_full(a) * tt_full(b)) <= 1e-12


def test_single_fourier_modes_multiply_to_one_mode():
    L = 10
    x = np.arange(2 ** L) / 2 ** L
    a = exp_mode_tt(0.7 - 0.2j, _site_angles([5], L, 1, "1d", 2 * np.pi))
    b = exp_mode_tt(1.1 + 0.4j, _site_angles([-3], L, 1, "1d", 2 * np.pi))
    r = oracle.aci([a, b], "mul", 1e-12, 16)
    exact = (0.7 - 0.2j) * (1.1 + 0.4j) * np.exp(2j * np.pi * 2 * x)
    assert max(r["ranks"]) == 1
    assert rel_err(tt_full(r["Y"]), exact) <= 1e-13


def test_times_one_is_identity_and_commutes():
    p = config_inputs(1)
    a, b = p["inputs"]
    one = [np.ones((1, 2, 1)) for _ in range(len(a))]
    r = oracle.aci([a, one], "mul", 1e-12, 64)
    assert rel_err(tt_full(r["Y"]), tt_full(a)) <= 1e-11
    r1 = oracle.aci([a, b], "mul", 1e-10, 64)
    r2 = oracle.aci([b, a], "mul", 1e-10, 64)
    assert r1["ranks"] == r2["ranks"]
    for y1, y2 in zip(r1["Y"], r2["Y"]):
        assert np.array_equal(y1, y2)
    r3 = oracle.aci([a, b], "mul_conj", 1e-10, 64)
    for y1, y3 in zip(r1["Y"], r3["Y"]):
        assert np.array_equal(y1, y3)


def test_interpolation_property_and_nesting():
    p = config_inputs(1)
    a, b = p["inputs"]
    r = oracle.aci([a, b], "mul", 1e-10, 64)
    L = len(a)
    J = r["J_sets"]
    for s in range(1, L - 1):  # right sets are nested after the final right-to-left sweep
        tails = set(J[s + 1])
        assert all(t[1:] in tails for t in J[s])
    # y equals f exactly on (sigma_0, j) for every j in J_1 (Sec. 2.5, CI-canonical form)
    pts = np.array([(s0,) + j for s0 in range(2) for j in J[1]])
    yv = tt_eval(r["Y"], pts)
    fv = tt_eval(a, pts) * tt_eval(b, pts)
    assert np.abs(yv - fv).max() <= 1e-13 * np.abs(fv).max()


@pytest.mark.parametrize("op", ["mul", "mul_conj", "abs2_mul", "affine"])
def test_ops_complex_dense(op):
    rng = np.random.default_rng(11)
    L = 8
    a = tt_random_uniform(rng, L, 2, 2, dtype=np.complex128, low=-1, high=1)
    b = tt_random_uniform(rng, L, 2, 2, dtype=np.complex128, low=-1, high=1)
    coef = (0.5 - 1j, 2.0, -1.5 + 0.25j, 0.75j)
    ins = [a] if op == "abs2_mul" else [a, b]
    r = oracle.aci(ins, op, 1e-14, 256, coef=coef)
    A, B = tt_full(a), tt_full(b)
    ref = {"mul": A * B, "mul_conj": A * np.conj(B), "abs2_mul": np.abs(A) ** 2 * A,
           "affine": coef[0] + coef[1] * A + coef[2] * B + coef[3] * A * B}[op]
    assert rel_err(tt_full(r["Y"]), ref) <= 1e-11


def test_gaussian_closed_form():
    g = json.load(open(os.path.join(GOLD, "paper_workloads.json")))["gaussians"]
    L = 16  # dense-checkable instead of the paper's 25
    for delta in g["deltas"]:
        gp, gm, x = gaussian_pair(L, g["w"], delta)
        h = np.exp(-x ** 2 / g["w"] ** 2 - delta ** 2 / (4 * g["w"] ** 2))
        r = oracle.aci([gp, gm], "mul", 1e-13, 64)
        err = np.abs(tt_full(r["Y"]) - h).max()
        assert err <= 100 * g["eps_float64_floor"], (delta, err)


def test_gaussian_error_falls_with_rank():
    g = json.load(open(os.path.join(GOLD, "paper_workloads.json")))["gaussians"]
    L = 16
    gp, gm, x = gaussian_pair(L, g["w"], 0.8)
    h = np.exp(-x ** 2 / g["w"] ** 2 - 0.8 ** 2 / (4 * g["w"] ** 2))
    errs = []
    for chi in (2, 4, 6, 8):
        r = oracle.aci([gp, gm], "mul", 0.0, chi, tol_kind="abs", maxiter=6)
        errs.append(np.abs(tt_full(r["Y"]) - h).max())
    assert errs[-1] < 1e-6 * errs[0] and errs[-1] < 1e-8, errs


def test_fourier_convolution_closed_form():
    g = json.load(open(os.path.join(GOLD, "paper_workloads.json")))["fourier"]
    K, L = 12, 16
    a, ia = fourier_paper_1d(5, K, L=L)
    b, ib = fourier_paper_1d(6, K, L=L)
    g1, g2 = ia["g"], ib["g"]
    h = np.array([sum(g1[k] * g2[q - k] for k in range(max(0, q - K), min(q, K) + 1))
                  for q in range(2 * K + 1)])  # reading of Eq. (fouriermultiplication)
    x = np.arange(2 ** L) / 2 ** L
    exact = np.exp(1j * np.outer(x, np.arange(2 * K + 1))) @ h
    r = oracle.aci([a, b], "mul", g["tau"], 64)
    err = np.abs(tt_full(r["Y"]) - exact).max()
    assert err <= 10 * g["tau"] * np.abs(exact).max(), err


def test_warm_start_from_previous_output():
    p = config_inputs(1)
    a, b = p["inputs"]
    r1 = oracle.aci([a, b], "mul", 1e-10, 64)
    r2 = oracle.aci([a, b], "mul", 1e-10, 64, init=r1["Y"])
    assert r2["iterations"] <= r1["iterations"]
    assert rel_err(tt_full(r2["Y"]), tt_full(a) * tt_full(b)) <= 1e-9


def test_three_and_four_inputs_reproduce_the_dense_product():
    """N > 2 inputs (Sec. 2.1, f of x^1..x^N): the product of three or four random low-rank TTs is
    reproduced exactly (its rank, the product of the input ranks, fits under the cap)."""
    rng = np.random.default_rng(31)
    for N, chi in ((3, 2), (4, 2)):
        ins = [tt_random_uniform(rng, 7, 2, chi, low=-1, high=1) for _ in range(N)]
        r = oracle.aci(ins, "mul", 1e-13, 64)
        exact = np.prod([tt_full(x) for x in ins], axis=0)
        assert np.abs(tt_full(r["Y"]) - exact).max() <= 1e-12 * np.abs(exact).max()
        assert max(r["ranks"]) <= chi ** N
