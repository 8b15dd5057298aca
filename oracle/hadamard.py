"""O(chi^4) Kronecker-delta Hadamard product followed by SVD truncation (oracle side).

TEST INFRASTRUCTURE ONLY (see the package header).

Prior work computes x^1 (.) x^2 by attaching a Kronecker delta to one input and
contracting (Sec. 1, Sec. 2.9, Appendix A). Written out, the product TT has cores
C_s[:, sigma, :] = A_s[:, sigma, :] (x) B_s[:, sigma, :] (Kronecker product of the
core slices), which is exact with rank chi_A * chi_B, and is then rounded by SVD.
This is used where chi_A * chi_B stays small enough (<= ~1024) to form the exact
product; the rounding follows the standard TT-SVD (QR sweep left to right, truncated
SVDs right to left, Frobenius tolerance split evenly over the L-1 bonds).

Pinned by: the exact product against dense brute force (tests/test_oracle_hadamard.py)
and the truncation error against its Frobenius bound.
"""

import numpy as np


def hadamard_kron(A, B, conj_b: bool = False):
    """Exact TT of the elementwise product a * b (or a * conj(b)): Kronecker product of slices."""
    out = []
    for a, b in zip(A, B):
        if conj_b:
            b = np.conj(b)
        ra, d, ra2 = a.shape
        rb, _, rb2 = b.shape
        c = np.einsum("asb,csd->acsbd", a, b).reshape(ra * rb, d, ra2 * rb2)
        out.append(c)
    return out


def tt_round_svd(cores, max_rank=None, rel_tol=0.0):
    """TT rounding: QR left to right, then truncated SVDs right to left."""
    cores = [c.copy() for c in cores]
    L = len(cores)
    for s in range(L - 1):
        r, d, rr = cores[s].shape
        q, rm = np.linalg.qr(cores[s].reshape(r * d, rr))
        cores[s] = q.reshape(r, d, q.shape[1])
        cores[s + 1] = np.tensordot(rm, cores[s + 1], axes=(1, 0))
    nrm = np.linalg.norm(cores[-1])
    thr2 = (rel_tol * nrm) ** 2 / max(L - 1, 1)
    for s in range(L - 1, 0, -1):
        r, d, rr = cores[s].shape
        u, sv, vh = np.linalg.svd(cores[s].reshape(r, d * rr), full_matrices=False)
        keep = len(sv)
        if rel_tol > 0:
            tail = np.cumsum((sv ** 2)[::-1])[::-1]
            ok = np.nonzero(tail <= thr2)[0]
            if len(ok):
                keep = max(1, int(ok[0]))
        if max_rank is not None:
            keep = min(keep, int(max_rank))
        cores[s] = vh[:keep].reshape(keep, d, rr)
        cores[s - 1] = np.tensordot(cores[s - 1], u[:, :keep] * sv[:keep], axes=(2, 0))
    return cores
