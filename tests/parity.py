"""Whole-call parity of the CUDA path (aci_elementwise_ex through the C ABI) against the oracle.

Two comparisons, both driven by the pivot history the library records for every local update
(aci_stats.hist_*):

followed_parity (full search). The oracle runs Algorithm 1 again while following the GPU's
pivots wherever they are as valid as its own argmax: a followed pivot must lie within
``slack`` x S of the largest remaining Schur entry, and a followed rank must stop where the
stop test of Algorithm 2 holds within the same slack (reading R4: when two candidates differ by
less than the rounding of the Schur entries, several pivot sequences are correct). Every pivot of
every update is checked this way, at any size. Until the first update where the GPU's choice was
not the oracle's own argmax (``differ``), the followed run IS the plain oracle run, so the GPU
history equals the plain oracle's history there. With the same pivots the two sides do the same
arithmetic up to rounding, so ranks, iteration counts and final pivots must be identical and the
outputs must agree to 1e-12 of max|y|.

tie_aware_parity (rook search, where the oracle has no follow mode). Pivots and ranks of every
update are compared in sweep order up to the first update at which the oracle saw a near-tie
(a top-2 gap below thr x S); values are always compared: to 1e-12 of max|y| when no near-tie
occurred, else to 10 x tol x max|y| (several outputs are then correct, each within tolerance).
"""

import numpy as np

import oracle
from synthetic import tt_full, tt_eval

NEAR_TIE = 1e-12


def to_dev(tt):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in tt]


def to_np(tt):
    return [c.cpu().numpy() if hasattr(c, "cpu") else c for c in tt]


def update_order(L, iterations):
    """The local updates of a call in execution order, as (u, b) history keys."""
    order = [(0, s - 1) for s in range(L - 1, 0, -1)]
    for it in range(1, iterations + 1):
        order += [(1 + 2 * (it - 1), b) for b in range(L - 1)]
        order += [(2 + 2 * (it - 1), b) for b in range(L - 2, -1, -1)]
    return order


def _values(y, yref, points):
    if points is None:
        return tt_full(y), tt_full(yref)
    return tt_eval(y, points), tt_eval(yref, points)


def run_gpu(ctx, inputs, op, tol, max_rank, coef=None, **gpu_kw):
    ins = to_dev(inputs[0]), (to_dev(inputs[1]) if len(inputs) > 1 else None)
    got, info = ctx.elementwise(*ins, op=op, tol=tol, max_rank=max_rank, coef=coef, pivots=True, history=True,
                                **gpu_kw)
    return to_np(got), info


def followed_parity(ctx, inputs, op, tol, max_rank, *, coef=None, oracle_kw=None, gpu_kw=None, points=None,
                    slack=1e-12, vtol=1e-12, gpu=None):
    """Full-search parity (module docstring). ``points``: None for a dense comparison, else an
    integer array (npts x L) of grid points. ``gpu``: a (y, info) pair from run_gpu to reuse.
    Returns (y, info, ref) with ref the followed oracle run (ref["follow"] its report)."""
    oracle_kw = dict(oracle_kw or {})
    gpu_kw = dict(gpu_kw or {})
    y, info = gpu if gpu is not None else run_gpu(ctx, inputs, op, tol, max_rank, coef=coef, **gpu_kw)
    ref = oracle.aci(inputs, op, tol, max_rank, coef=coef, follow=info["history"], follow_slack=slack,
                     maxiter=gpu_kw.get("max_sweeps", 20), **oracle_kw)
    rep = ref["follow"]
    assert not rep["violations"], rep["violations"][:5]
    L = len(inputs[0])
    assert set(info["history"]) == set(update_order(L, info["iterations"])), "history covers every update"
    assert rep["updates"] == len(info["history"])
    assert info["iterations"] == ref["iterations"]
    assert info["ranks"] == ref["ranks"]
    for b in range(L - 1):
        assert info["pivot_rows"][b] == [int(v) for v in ref["I_pos"][b]], b
        assert info["pivot_cols"][b] == [int(v) for v in ref["J_pos"][b]], b
    yg, yr = _values(y, ref["Y"], points)
    assert np.abs(yg - yr).max() <= vtol * np.abs(yr).max(), np.abs(yg - yr).max() / np.abs(yr).max()
    return y, info, ref


def first_tie(log, L, thr=NEAR_TIE):
    """Position in update_order of the first sweep update with a near-tie (None if there is none)."""
    order = update_order(L, max((e["u"] - 1) // 2 + 1 for e in log) if log else 0)
    tied = {(e["u"], e["bond"]) for e in log if len(e["best"]) and ((e["best"] - e["second"]) / e["S"]).min() < thr}
    for i, key in enumerate(order):
        if key in tied:
            return i
    return None


def tie_aware_parity(ctx, inputs, op, tol, max_rank, *, coef=None, oracle_kw=None, gpu_kw=None, points=None):
    """Rook-search parity (module docstring). Returns (y, info, ref, tie) with tie the position
    (in update order) of the oracle's first near-tie, None if none."""
    oracle_kw = dict(oracle_kw or {})
    gpu_kw = dict(gpu_kw or {})
    y, info = run_gpu(ctx, inputs, op, tol, max_rank, coef=coef, **gpu_kw)
    ref = oracle.aci(inputs, op, tol, max_rank, coef=coef, record=True, maxiter=gpu_kw.get("max_sweeps", 20),
                     **oracle_kw)
    L = len(inputs[0])
    for e, (u, b) in zip(ref["log"], [k for k in update_order(L, ref["iterations"]) if k[0] > 0]):
        e["u"] = u
    tie = first_tie(ref["log"], L)
    order = update_order(L, min(info["iterations"], ref["iterations"]))
    upto = order if tie is None else order[:tie]
    for key in upto:
        gr, gc = info["history"][key]
        rr, rc = ref["history"][key]
        assert list(gr) == [int(v) for v in rr] and list(gc) == [int(v) for v in rc], key
    yg, yr = _values(y, ref["Y"], points)
    scale = np.abs(yr).max()
    if tie is None:
        assert info["ranks"] == ref["ranks"]
        assert info["iterations"] == ref["iterations"]
        assert np.abs(yg - yr).max() <= 1e-12 * scale
    else:
        assert np.abs(yg - yr).max() <= 10 * tol * scale
    return y, info, ref, tie
