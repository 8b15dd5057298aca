"""Plain tensor-train utilities for building and checking inputs.

A TT is a list of cores; core ``s`` has shape ``(r_s, d_s, r_{s+1})`` with
``r_0 = r_L = 1`` (Sec. 2.1: x_{sigma_1..sigma_L} as a product of core slices).
Values are ``x[sigma] = X_0[:, sigma_0, :] @ X_1[:, sigma_1, :] @ ... @ X_{L-1}[:, sigma_{L-1}, :]``.
"""

from __future__ import annotations

import numpy as np

TT = list  # list of np.ndarray cores (r_l, d_l, r_r)


def tt_ranks(cores) -> list[int]:
    return [int(cores[0].shape[0])] + [int(c.shape[2]) for c in cores]


def tt_full(cores) -> np.ndarray:
    """Dense tensor of a TT, flattened with site 0 as the most significant index."""
    v = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])
    for c in cores[1:]:
        r, d, rr = c.shape
        v = (v @ c.reshape(r, d * rr)).reshape(-1, rr)
    return v.reshape(-1)


def tt_eval(cores, sigma: np.ndarray) -> np.ndarray:
    """Values of a TT at multi-indices ``sigma`` (shape (P, L)), one product chain per point:
    at each site the points are grouped by their local index, so each group is one matrix product."""
    sigma = np.asarray(sigma)
    P = sigma.shape[0]
    dtype = np.result_type(*[c.dtype for c in cores])
    v = np.ones((P, 1), dtype=dtype)
    for s, c in enumerate(cores):
        out = np.empty((P, c.shape[2]), dtype=dtype)
        for x in range(c.shape[1]):
            m = sigma[:, s] == x
            if m.any():
                out[m] = v[m] @ c[:, x, :]
        v = out
    return v[:, 0]


def tt_block_sum(tts) -> list:
    """Exact TT of a sum of TTs: cores are block diagonal, ranks add (first/last are concatenated)."""
    L = len(tts[0])
    dtype = np.result_type(*[c.dtype for t in tts for c in t])
    out = []
    for s in range(L):
        ds = tts[0][s].shape[1]
        rl = [t[s].shape[0] for t in tts]
        rr = [t[s].shape[2] for t in tts]
        if L == 1:
            core = sum(t[0] for t in tts).astype(dtype)
        elif s == 0:
            core = np.concatenate([t[s] for t in tts], axis=2).astype(dtype)
        elif s == L - 1:
            core = np.concatenate([t[s] for t in tts], axis=0).astype(dtype)
        else:
            core = np.zeros((sum(rl), ds, sum(rr)), dtype=dtype)
            a = b = 0
            for t, x, y in zip(tts, rl, rr):
                core[a:a + x, :, b:b + y] = t[s]
                a += x
                b += y
        out.append(core)
    return out


def _left_orthogonalize(cores):
    cores = [c.copy() for c in cores]
    for s in range(len(cores) - 1):
        r, d, rr = cores[s].shape
        q, rmat = np.linalg.qr(cores[s].reshape(r * d, rr))
        cores[s] = q.reshape(r, d, q.shape[1])
        nxt = cores[s + 1]
        cores[s + 1] = np.tensordot(rmat, nxt, axes=(1, 0))
    return cores


def tt_svd_round(cores, max_rank: int | None = None, rel_tol: float = 0.0):
    """TT rounding: left-orthogonalise by QR, then truncated SVDs right to left.

    Each bond keeps at most ``max_rank`` singular values and drops the tail whose
    squared sum stays below ``(rel_tol * ||x||_F)^2 / (L-1)``.
    """
    L = len(cores)
    cores = _left_orthogonalize(cores)
    norm = np.linalg.norm(cores[-1])
    thr2 = (rel_tol * norm) ** 2 / max(L - 1, 1)
    for s in range(L - 1, 0, -1):
        r, d, rr = cores[s].shape
        u, sv, vh = np.linalg.svd(cores[s].reshape(r, d * rr), full_matrices=False)
        keep = len(sv)
        if rel_tol > 0:
            tail = np.cumsum((sv ** 2)[::-1])[::-1]  # tail[i] = sum_{j>=i} sv_j^2
            ok = np.nonzero(tail <= thr2)[0]
            if len(ok):
                keep = max(1, int(ok[0]))
        if max_rank is not None:
            keep = min(keep, int(max_rank))
        u, sv, vh = u[:, :keep], sv[:keep], vh[:keep]
        cores[s] = vh.reshape(keep, d, rr)
        cores[s - 1] = np.tensordot(cores[s - 1], u * sv, axes=(2, 0))
    return cores


def tt_from_dense(v: np.ndarray, dims, max_rank=None, rel_tol=0.0):
    """TT-SVD of a dense vector with site dims ``dims`` (site 0 most significant)."""
    cores = []
    rest = np.asarray(v).reshape(1, -1)
    L = len(dims)
    r = 1
    for s in range(L - 1):
        m = rest.reshape(r * dims[s], -1)
        u, sv, vh = np.linalg.svd(m, full_matrices=False)
        keep = int(np.sum(sv > sv[0] * 1e-15)) if sv[0] > 0 else 1
        keep = max(keep, 1)
        if max_rank is not None:
            keep = min(keep, max_rank)
        cores.append(u[:, :keep].reshape(r, dims[s], keep))
        rest = sv[:keep, None] * vh[:keep]
        r = keep
    cores.append(rest.reshape(r, dims[-1], 1))
    if rel_tol > 0 or max_rank is not None:
        cores = tt_svd_round(cores, max_rank=max_rank, rel_tol=rel_tol)
    return cores


def tt_random_uniform(rng: np.random.Generator, L: int, d: int, chi: int,
                      dtype=np.float64, low=0.0, high=1.0):
    """TT with cores drawn uniformly from [low, high) (Sec. 3.3), bonds min(chi, d^s, d^(L-s))."""
    ranks = [1] + [min(chi, d ** s, d ** (L - s)) for s in range(1, L)] + [1]
    cores = []
    for s in range(L):
        shape = (ranks[s], d, ranks[s + 1])
        c = rng.uniform(low, high, size=shape)
        if np.iscomplexobj(np.zeros(1, dtype=dtype)):
            c = c + 1j * rng.uniform(low, high, size=shape)
        cores.append(c.astype(dtype))
    return cores


def quantics_points(sigma: np.ndarray, bits_per_site: int = 1, ndim: int = 1,
                    interleaved: bool = False) -> np.ndarray:
    """Grid coordinates of multi-indices (Eq. (quanticsrep)), site 0 = most significant bit.

    1D: x = sum_l 2^-l sigma_l. 2D interleaved: sites alternate (x_1, y_1, x_2, y_2, ...).
    Fused d=8: sigma_l = 4 b_x + 2 b_y + b_z at site l.
    Returns an array of shape (P, ndim) in [0, 1).
    """
    sigma = np.asarray(sigma, dtype=np.int64)
    P, L = sigma.shape
    if ndim == 1:
        w = 0.5 ** np.arange(1, L + 1)
        return (sigma * w).sum(axis=1)[:, None]
    if interleaved:
        nb = L // ndim
        out = np.zeros((P, ndim))
        for a in range(ndim):
            bits = sigma[:, a::ndim]
            out[:, a] = (bits * 0.5 ** np.arange(1, nb + 1)).sum(axis=1)
        return out
    # fused: each site carries one bit of every dimension, MSB of sigma = first dimension
    out = np.zeros((P, ndim))
    for a in range(ndim):
        bits = (sigma >> (ndim - 1 - a)) & 1
        out[:, a] = (bits * 0.5 ** np.arange(1, L + 1)).sum(axis=1)
    return out
