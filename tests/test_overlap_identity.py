"""The identity the overlapped sweep schedule rests on, with the index maps its gathers use
(aci_opts.sweep_overlap; CPU, numpy). For one bond of a two-input product f(a, b):

Left to right (Algorithm 5's left frame, Eq. (pifromframes)): with LX_b = (rows prow of
LX_{b-1}) X_b, Pi = f(LX_b XR_{b+1}) equals the rows of f(Q XR_{b+1}), Q = LX_{b-1} X_b over every
row of Pi[b-1], taken by blocks of d_b rows: row i d_b + s of Pi is row prow[i] d_b + s of the full
block. LX_b itself is rows prow of Q (each a d_b r_{b+1} row).

Right to left (the right frame): with XR_{b+1} = X_{b+1} (columns pcol of XR_{b+2}), Pi equals the
columns of f(LX_b P), P = X_{b+1} XR_{b+2} over every column of Pi[b+1], taken per sigma_{b+1}
slab: column s chi + j of Pi is column s N + pcol[j] of the full block (N = d_{b+2} chi_{b+3}, the
columns of Pi[b+1]); XR_{b+1} is the same columns of P.

The contractions are plain matmuls here; the identity is exact up to rounding, so a mistake in
an index map (block size, slab stride, row vs column) shows as an O(1) difference."""

import numpy as np
import pytest


def f(u, v):
    return u * v


def gather_rows_blocked(M, idx, blk):
    """Rows idx[r // blk] * blk + r % blk of M, for r < len(idx) * blk."""
    r = np.arange(len(idx) * blk)
    return M[np.asarray(idx)[r // blk] * blk + r % blk]


def gather_cols_slabs(M, idx, blk, stride, nslabs):
    """Columns (c // blk) * stride + idx[c % blk] of M, for c < nslabs * blk."""
    c = np.arange(nslabs * blk)
    return M[:, (c // blk) * stride + np.asarray(idx)[c % blk]]


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("cplx", [False, True])
def test_left_to_right_gather_identity(seed, cplx):
    rng = np.random.default_rng(seed)
    dt = np.complex128 if cplx else np.float64
    rnd = (lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)) if cplx else (lambda *s: rng.standard_normal(s))
    chi_prev, d_prev, d_b, d_next, chi_b, chi_next2 = 3, 2, int(rng.integers(2, 5)), 2, 4, 5
    r_b, r_next = 3, 4  # input bond ranks r_b (into site b) and r_{b+1}
    ins = []
    for _ in range(2):
        LXprev = rnd(chi_prev * d_prev, r_b).astype(dt)               # LX_{b-1}: (chi_{b-1} d_{b-1}) x r_b
        Xb = rnd(r_b, d_b, r_next).astype(dt)                         # X_b: r_b x d_b x r_{b+1}
        XRnext = rnd(r_next, d_next * chi_next2).astype(dt)           # XR_{b+1}: r_{b+1} x (d_{b+1} chi_{b+2})
        ins.append((LXprev, Xb, XRnext))
    prow = rng.choice(chi_prev * d_prev, size=chi_b, replace=False)   # pivots of bond b-1 (rows of Pi[b-1])
    # plain: LX_b = rows prow of LX_{b-1}, times X_b, as (chi_b d_b) x r_{b+1}; then Pi
    prods = []
    for LXprev, Xb, XRnext in ins:
        LXb = (LXprev[prow] @ Xb.reshape(r_b, d_b * r_next)).reshape(chi_b * d_b, r_next)
        prods.append(LXb @ XRnext)
    Pi = f(*prods)
    # overlapped: Q over every row of Pi[b-1], the full block, then the blocked row gather
    full = []
    Qs = []
    for LXprev, Xb, XRnext in ins:
        Q = LXprev @ Xb.reshape(r_b, d_b * r_next)                     # (chi_{b-1} d_{b-1}) x (d_b r_{b+1})
        Qs.append(Q)
        full.append(Q.reshape(chi_prev * d_prev * d_b, r_next) @ XRnext)
    Pfull = f(*full)
    Pi_gathered = gather_rows_blocked(Pfull, prow, d_b)
    assert np.abs(Pi_gathered - Pi).max() <= 1e-13 * np.abs(Pi).max()
    # LX_b is the plain row gather of Q
    LXb0 = (ins[0][0][prow] @ ins[0][1].reshape(r_b, d_b * r_next))
    assert np.abs(Qs[0][prow] - LXb0).max() <= 1e-13 * np.abs(LXb0).max()


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("cplx", [False, True])
def test_right_to_left_gather_identity(seed, cplx):
    rng = np.random.default_rng(100 + seed)
    dt = np.complex128 if cplx else np.float64
    rnd = (lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)) if cplx else (lambda *s: rng.standard_normal(s))
    chi_b, d_b = 3, 2
    d_b1, d_b2, chi_b3, chi_b2 = int(rng.integers(2, 5)), 2, 3, 4
    r_b1, r_b2 = 3, 4          # input ranks r_{b+1}, r_{b+2}
    N = d_b2 * chi_b3          # columns of Pi[b+1]
    ins = []
    for _ in range(2):
        LXb = rnd(chi_b * d_b, r_b1).astype(dt)                       # LX_b: (chi_b d_b) x r_{b+1}
        Xb1 = rnd(r_b1, d_b1, r_b2).astype(dt)                        # X_{b+1}
        XRb2 = rnd(r_b2, N).astype(dt)                                # XR_{b+2}: r_{b+2} x (d_{b+2} chi_{b+3})
        ins.append((LXb, Xb1, XRb2))
    pcol = rng.choice(N, size=chi_b2, replace=False)                  # pivots of bond b+1 (columns of Pi[b+1])
    prods = []
    XRs = []
    for LXb, Xb1, XRb2 in ins:
        XRb1 = (Xb1.reshape(r_b1 * d_b1, r_b2) @ XRb2[:, pcol]).reshape(r_b1, d_b1 * chi_b2)
        XRs.append(XRb1)
        prods.append(LXb @ XRb1)
    Pi = f(*prods)
    full = []
    Ps = []
    for LXb, Xb1, XRb2 in ins:
        P = (Xb1.reshape(r_b1 * d_b1, r_b2) @ XRb2).reshape(r_b1, d_b1 * N)   # r_{b+1} x (d_{b+1} N)
        Ps.append(P)
        full.append(LXb @ P)
    Pfull = f(*full)
    Pi_gathered = gather_cols_slabs(Pfull, pcol, chi_b2, N, d_b1)
    assert np.abs(Pi_gathered - Pi).max() <= 1e-13 * np.abs(Pi).max()
    XR_gathered = gather_cols_slabs(Ps[0], pcol, chi_b2, N, d_b1)
    assert np.abs(XR_gathered - XRs[0]).max() <= 1e-13 * np.abs(XRs[0]).max()


def test_a_wrong_map_is_caught():
    """A plain (unblocked) row gather in place of the blocked one is O(1) off."""
    rng = np.random.default_rng(7)
    M = rng.standard_normal((12, 5))
    idx = np.array([4, 0, 2])
    good = gather_rows_blocked(M, idx, 2)
    bad = M[np.repeat(idx, 2)]
    assert np.abs(good - bad).max() > 0.1
