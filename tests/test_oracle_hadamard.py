"""Pins for the oracle's Kronecker-delta Hadamard product and SVD rounding (Sec. 2.9, App. A)."""

import numpy as np

from oracle import hadamard_kron, tt_round_svd
import oracle
from synthetic import tt_full, tt_random_uniform, config_inputs


def test_kron_product_exact_dense():
    rng = np.random.default_rng(1)
    a = tt_random_uniform(rng, 7, 2, 3, dtype=np.complex128, low=-1, high=1)
    b = tt_random_uniform(rng, 7, 2, 4, dtype=np.complex128, low=-1, high=1)
    A, B = tt_full(a), tt_full(b)
    assert np.abs(tt_full(hadamard_kron(a, b)) - A * B).max() <= 1e-13 * np.abs(A * B).max()
    assert np.abs(tt_full(hadamard_kron(a, b, conj_b=True)) - A * np.conj(B)).max() <= 1e-13 * np.abs(A * B).max()


def test_rounding_error_within_frobenius_bound():
    rng = np.random.default_rng(2)
    a = tt_random_uniform(rng, 9, 2, 4, low=-1, high=1)
    b = tt_random_uniform(rng, 9, 2, 4, low=-1, high=1)
    c = hadamard_kron(a, b)
    full = tt_full(c)
    for tol in (1e-2, 1e-5, 1e-9):
        r = tt_round_svd(c, rel_tol=tol)
        assert np.linalg.norm(tt_full(r) - full) <= tol * np.linalg.norm(full) * (1 + 1e-8)


def test_aci_agrees_with_kron_svd_within_tolerance():
    p = config_inputs(1)
    a, b = p["inputs"]
    r = oracle.aci([a, b], "mul", 1e-10, 64)
    ref = tt_full(tt_round_svd(hadamard_kron(a, b), rel_tol=1e-13))
    y = tt_full(r["Y"])
    assert np.abs(y - ref).max() <= 20 * 1e-10 * np.abs(ref).max()
