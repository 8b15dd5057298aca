"""Plain CPU restatement of alternating cross interpolation (ACI), Appendix B.

TEST INFRASTRUCTURE ONLY (see the package header): imported by tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg, never by the library.

Everything is FP64 / complex128 numpy, written in the order and notation of the
paper's Algorithms 1-5, with 0-based sites s = 0..L-1 (the paper's site l = s + 1).
Index sets are kept as lists of multi-index tuples, exactly as defined in Sec. 2.5:
I_s holds tuples (sigma_0..sigma_s) and J_s holds tuples (sigma_s..sigma_{L-1}).
Frames are rebuilt from the index sets with Algorithm 5 at every step (no caching).

Readings of places where the paper is silent or garbled:
  R1  tol is relative by default: tau = tol * S, S the running max |Pi| over all Pi
      blocks formed so far in the call; tol_kind="abs" gives Alg. 1's absolute tau.
      The initial-guess CI uses tau = tol * max|M| of its own matrix (or tol for "abs").
  R2  Alg. 2 stops *before* accepting a pivot with |pivot| <= tau, or once chi_hat pivots
      are taken; epsilon is the magnitude of the first rejected pivot (the largest
      remaining Schur entry), 0 when the Schur block is empty.
  R3  Alg. 2's second swap exchanges J_j (not J_i) with J_chi; Alg. 3's L_{I,1:n} and
      U_{1:m,J} are the k x k blocks L_{I,1:k}, U_{1:k,J}.  L and U are unit triangular:
      L_{rp} = S_{rp}/S_{pp}, U_{pc} = S_{pc}/S_{pp} from the in-place elimination.
  R4  At least one pivot is always taken. Pivot search maximises |v| (real) or
      re^2 + im^2 (complex, each product and the sum rounded separately); exact ties
      go to the lowest original linear index row * n + col. A zero pivot (all-zero
      block) gives unit L/U columns, D = 0, and D^-1 is read as 0.
  R5  Alg. 1 writes I_l and J_{l+1} at bond l (Sec. 2.6 prose says I_{l+1}, J_l).
  R6  The output is y = T_0 P_0^-1 T_1 P_1^-1 ... T_{L-1} from the last right-to-left
      sweep: Y_0 = A_0 = L L_I^-1 of bond 0, Y_s = B_{s-1} P_s^-1 with
      B_{s-1} = L_I D U of bond s-1 and P_s = L_I D U_J of bond s, Y_{L-1} = B_{L-2}.
  R7  The CI-canonicalisation of Y^init uses CI "right", keeps J_l, and multiplies
      A = L D U_J into Y_{l-1}.
  R8  maxiter defaults to 20; epsilon of an iteration is the max over both half-sweeps;
      ranks are compared with those at the end of the previous iteration (after the
      initial CI for the first). A second stop: an iteration that reproduces every J
      set of the previous one is a fixed point (the next sweep would repeat it exactly).
  R9  Y^init is the counter-based SplitMix64 TT of oracle.rng with ranks
      min(chi_hat, min_n r^n_s, prod_{t<s} d_t, prod_{t>=s} d_t), unless the caller passes one.
  R10 (reserved)
  R11 Rook search (pivot_mode="rook"; not written in the paper, whose O(d chi'^3) cost per
      update in App. A fits a partial search): the residual R_p = M - sum_{q<p} L_q D_q U_q
      is formed lazily, one column or row at a time. Step 0 starts from the column of the
      global argmax of |M|; step p >= 1 from the column of the largest residual of the
      previous pivot row (before its elimination) among unused columns. From column c0:
      r1 = argmax_r |R(r,c0)|, c1 = argmax_c |R(r1,c)|; c1 == c0 accepts (r1, c0); else
      r2 = argmax_r |R(r,c1)|; r2 == r1 accepts (r1, c1); else (r2, c1) is accepted after
      the fourth hop. Searches run over unused rows / columns with the key and tie rule of
      R4 (lowest index). The pivot value is taken from the column evaluation; L's column is
      the residual column over the pivot, U's row the residual row over the pivot. The stop
      test and epsilon are those of R2 with the rook pivot in place of the block maximum.

Parity pins (tests/test_oracle_*.py): LDU against an independent complete-pivoting LU
and brute-force residual identities; CI factors against exact interpolation on the
pivot cross; ACI against dense brute force on small grids, closed-form Fourier and
Gaussian products (Eqs. (gaussians), (fouriermultiplication)), exact low-rank products,
commutativity and the interpolation property of the CI-canonical form.
"""

from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from .rng import random_tt_counter

# ---------------------------------------------------------------- elementwise f (Sec. 2.1)

OPS = ("mul", "mul_conj", "abs2_mul", "affine")


def apply_op(op: str, xs, coef=None):
    """f(x^1, ..., x^N) entrywise: a*b, a*conj(b), |a|^2 a, or c0 + c1 a + c2 b + c3 a b; for
    N > 2 inputs "mul" is the product of all of them, taken left to right."""
    a = xs[0]
    b = xs[1] if len(xs) > 1 else None
    if op == "mul":
        out = a * b
        for x in xs[2:]:
            out = out * x
        return out
    if op == "mul_conj":
        return a * np.conj(b)
    if op == "abs2_mul":
        if np.iscomplexobj(a):
            return (a.real * a.real + a.imag * a.imag) * a
        return (a * a) * a
    if op == "affine":
        c0, c1, c2, c3 = coef
        return c0 + c1 * a + c2 * b + c3 * (a * b)
    raise ValueError(op)


def magnitude(v):
    """|v|: fabs for real, sqrt(re*re + im*im) for complex (no fused operations)."""
    v = np.asarray(v)
    if np.iscomplexobj(v):
        return np.sqrt(v.real * v.real + v.imag * v.imag)
    return np.abs(v)


def pivot_key(v):
    """Quantity maximised by the pivot search (R4)."""
    v = np.asarray(v)
    if np.iscomplexobj(v):
        return v.real * v.real + v.imag * v.imag
    return np.abs(v)


# ---------------------------------------------------------------- Algorithm 2: LDU (prrLU)

def ldu(M, tau: float, chimax: int, follow=None, slack: float = 0.0):
    """Algorithm 2: in-place LDU with full-search pivoting (readings R2-R4).

    ``follow`` = (rows, cols): another implementation's pivots (original positions, in pivot
    order) to take instead of this function's own argmax wherever they are an equally valid
    choice (R4: when two candidates' magnitudes differ by less than the rounding of the Schur
    entries, either is correct). A followed pivot must lie within ``slack`` (absolute magnitude)
    of the largest remaining one, and the followed rank must stop where the stop test allows it
    within ``slack`` of tau; each breach is appended to the result's ``violations`` (and this
    function's own choice is taken there). ``differ`` counts the steps where a followed pivot
    was not this function's own argmax.

    Returns a dict with
      L  (m x k) unit lower triangular in pivot order, rows in M's original row order,
      D  (k,)   pivots,
      U  (k x n) unit upper triangular in pivot order, columns in M's original order,
      I, J      pivot row / column positions of M in pivot order,
      eps       error estimate, k the rank,
      best, second  per accepted pivot: its magnitude and the next-largest candidate's.
    """
    S = np.array(M, copy=True)
    m, n = S.shape
    I = np.arange(m)  # I[pos] = original row now at position pos
    J = np.arange(n)
    chi = 0
    eps = 0.0
    best_list, second_list = [], []
    violations, differ = [], 0
    kfollow = len(follow[0]) if follow is not None else None
    while True:
        if chi == min(m, n):
            eps = 0.0
            if follow is not None and kfollow != chi:
                violations.append((chi, "followed rank differs at an exhausted block"))
            break
        sub = S[chi:, chi:]
        key = pivot_key(sub)
        kbest = key.max()
        where = np.argwhere(key == kbest)
        lin = I[chi + where[:, 0]] * n + J[chi + where[:, 1]]
        i, j = where[int(np.argmin(lin))] + chi
        piv = S[i, j]
        mag = float(magnitude(piv))
        stop = chi == chimax or (chi >= 1 and mag <= tau)
        if follow is not None:
            if chi >= kfollow:  # the other side stopped here: allowed if the stop test holds within slack
                if not (stop or mag <= tau + slack):
                    violations.append((chi, f"followed rank stops early: best {mag:.17g} > tau {tau:.17g}"))
                eps = mag
                break
            # the other side accepted a pivot: allowed unless the stop test holds beyond slack
            if chi == chimax or (chi >= 1 and mag < tau - slack):
                violations.append((chi, "followed rank continues past the stop test"))
            else:
                pr = np.flatnonzero(I[chi:] == follow[0][chi])
                pc = np.flatnonzero(J[chi:] == follow[1][chi])
                if len(pr) != 1 or len(pc) != 1:
                    violations.append((chi, "followed pivot is in a used row or column"))
                else:
                    fi, fj = pr[0] + chi, pc[0] + chi
                    fmag = float(magnitude(S[fi, fj]))
                    if fmag < mag - slack:
                        violations.append((chi, f"followed pivot {fmag:.17g} below the maximum {mag:.17g}"))
                    elif (fi, fj) != (i, j):
                        differ += 1
                        i, j, piv, mag = fi, fj, S[fi, fj], fmag
            stop = False
        if stop:
            eps = mag
            break
        flat = key.reshape(-1).copy()
        flat[(i - chi) * (n - chi) + (j - chi)] = -np.inf
        sec = float(flat.max()) if flat.size > 1 else -np.inf
        if np.iscomplexobj(S) and sec > -np.inf:
            sec = float(np.sqrt(sec))
        best_list.append(mag)
        second_list.append(sec)
        # swap the pivot to position (chi, chi) in M, and in I and J (R3: J_j, not J_i)
        S[[i, chi], :] = S[[chi, i], :]
        S[:, [j, chi]] = S[:, [chi, j]]
        I[[i, chi]] = I[[chi, i]]
        J[[j, chi]] = J[[chi, j]]
        # Schur complement (Gaussian elimination step)
        if piv != 0:
            l = S[chi + 1:, chi] / S[chi, chi]
            S[chi + 1:, chi + 1:] -= np.outer(l, S[chi, chi + 1:])
        chi += 1
    k = chi
    D = np.array([S[p, p] for p in range(k)], dtype=S.dtype)
    Lp = np.zeros((m, k), dtype=S.dtype)
    Up = np.zeros((k, n), dtype=S.dtype)
    for p in range(k):
        if D[p] != 0:
            Lp[p + 1:, p] = S[p + 1:, p] / D[p]
            Up[p, p + 1:] = S[p, p + 1:] / D[p]
        Lp[p, p] = 1
        Up[p, p] = 1
    L = np.zeros_like(Lp)
    U = np.zeros_like(Up)
    L[I, :] = Lp  # undo the row permutation: L[I[pos]] = Lp[pos]
    U[:, J] = Up
    return dict(L=L, D=D, U=U, I=I[:k].copy(), J=J[:k].copy(), eps=eps, k=k,
                best=np.array(best_list), second=np.array(second_list), violations=violations,
                differ=differ)


def _argmax_free(key, free):
    """Index of the largest key among free entries (ties to the lowest index), its key and the
    next-largest free key (-inf if none)."""
    k = np.where(free, key, -np.inf)
    i = int(np.argmax(k))  # first occurrence: the lowest index among exact ties
    rest = k.copy()
    rest[i] = -np.inf
    return i, float(k[i]), float(rest.max()) if rest.size > 1 else -np.inf


def ldu_rook(M, tau: float, chimax: int):
    """Rook-search prrLU (reading R11): the factors, stop test and outputs of ldu() with each
    pivot found by alternating row and column searches of the lazily formed residual."""
    M = np.array(M, copy=True)
    m, n = M.shape
    cplx = np.iscomplexobj(M)
    kcap = min(m, n, chimax)
    L = np.zeros((m, kcap), dtype=M.dtype)
    U = np.zeros((kcap, n), dtype=M.dtype)
    D = np.zeros(kcap, dtype=M.dtype)
    free_r = np.ones(m, dtype=bool)
    free_c = np.ones(n, dtype=bool)
    I, J = [], []
    best_list, second_list = [], []
    eps = 0.0
    p = 0
    c_next = None

    def mag_of_key(k):
        if not np.isfinite(k):
            return k
        return np.sqrt(k) if cplx else k

    def resid_col(c):
        return M[:, c] - L[:, :p] @ (D[:p] * U[:p, c])

    def resid_row(r):
        return M[r, :] - (L[r, :p] * D[:p]) @ U[:p, :]

    while True:
        if p == min(m, n):
            eps = 0.0
            break
        gaps = []
        if p == 0:  # the column of the global argmax of |M| (R4 ties: lowest row * n + col)
            key = pivot_key(M)
            flat = key.reshape(-1)
            c0 = int(np.argmax(flat)) % n
            srt = np.sort(flat)
            if flat.size > 1:
                gaps.append(mag_of_key(srt[-1]) - mag_of_key(srt[-2]))
        else:
            c0 = c_next
        col = resid_col(c0)
        r1, k1, k1b = _argmax_free(pivot_key(col), free_r)
        row = resid_row(r1)
        c1, k2, k2b = _argmax_free(pivot_key(row), free_c)
        gaps += [mag_of_key(k1) - mag_of_key(k1b), mag_of_key(k2) - mag_of_key(k2b)]
        if c1 == c0:
            r, c = r1, c0
        else:
            col = resid_col(c1)
            r2, k3, k3b = _argmax_free(pivot_key(col), free_r)
            gaps.append(mag_of_key(k3) - mag_of_key(k3b))
            if r2 == r1:
                r, c = r1, c1
            else:
                r, c = r2, c1
                row = resid_row(r2)
        piv = col[r]
        mag = float(magnitude(piv))
        if p == chimax or (p >= 1 and mag <= tau):
            eps = mag
            break
        if piv != 0:
            L[:, p] = np.where(free_r, col / piv, 0)
            U[p, :] = np.where(free_c, row / piv, 0)
        L[r, p] = 1
        U[p, c] = 1
        D[p] = piv
        free_r[r] = False
        free_c[c] = False
        I.append(r)
        J.append(c)
        if free_c.any():  # the next start column: largest residual of this pivot row (R11)
            c_next, kn, knb = _argmax_free(pivot_key(row), free_c)
            gaps.append(mag_of_key(kn) - mag_of_key(knb))
        best_list.append(mag)
        g = [x for x in gaps if np.isfinite(x)]
        second_list.append(mag - (min(g) if g else np.inf))
        p += 1
    k = p
    return dict(L=L[:, :k].copy(), D=D[:k].copy(), U=U[:k, :].copy(), I=np.array(I, dtype=np.int64),
                J=np.array(J, dtype=np.int64), eps=eps, k=k, best=np.array(best_list),
                second=np.array(second_list))


PIVOT_MODES = ("full", "rook")


def factorise(M, tau: float, chimax: int, pivot_mode: str = "full", follow=None, slack: float = 0.0):
    """Algorithm 2 with the full search, or the rook search of reading R11."""
    if pivot_mode == "full":
        return ldu(M, tau, chimax, follow, slack)
    if follow is not None:
        raise ValueError("following another implementation's pivots is defined for the full search")
    if pivot_mode == "rook":
        return ldu_rook(M, tau, chimax)
    raise ValueError(pivot_mode)


# ---------------------------------------------------------------- Algorithm 3: CI

def _inv_diag(D):
    out = np.zeros_like(D)
    nz = D != 0
    out[nz] = 1.0 / D[nz]
    return out


def crossinterpolate(M, tau: float, chimax: int, leftorright: str = "right", pivot_mode: str = "full",
                     follow=None, slack: float = 0.0):
    """Algorithm 3: A, B with A @ B = L D U ~ M; "left" puts P^-1 into A, "right" into B."""
    f = factorise(M, tau, chimax, pivot_mode, follow, slack)
    L, D, U, I, J = f["L"], f["D"], f["U"], f["I"], f["J"]
    if leftorright == "left":
        LI = L[I, :]  # k x k unit lower
        # A = L LI^-1  <=>  LI^T A^T = L^T
        A = solve_triangular(LI.T, L.T, lower=False, unit_diagonal=True).T
        B = LI @ (D[:, None] * U)
    else:
        UJ = U[:, J]  # k x k unit upper
        A = L @ (D[:, None] * UJ)
        B = solve_triangular(UJ, U, lower=False, unit_diagonal=True)
    f.update(A=A, B=B)
    return f


# ---------------------------------------------------------------- Algorithm 4: local update

def localupdate(Pi, tau: float, chimax: int, leftorright: str, pivot_mode: str = "full",
                follow=None, slack: float = 0.0):
    """Algorithm 4: reshape Pi[alpha, s, s', beta] to M[(alpha, s), (s', beta)] and factorise."""
    a, d1, d2, b = Pi.shape
    M = Pi.reshape(a * d1, d2 * b)
    f = crossinterpolate(M, tau, chimax, leftorright, pivot_mode, follow, slack)
    k = f["k"]
    f["Y"] = f["A"].reshape(a, d1, k)
    f["Y2"] = f["B"].reshape(k, d2, b)
    return f


# ---------------------------------------------------------------- Algorithm 5: frames

def leftframe(X, Lf, Iprev, Inew):
    """Algorithm 5 (left): L'_{(i,s),beta} = L_{i,gamma} X^s_{gamma,beta}, then keep rows Inew."""
    d = X.shape[1]
    Lp = np.einsum("ig,gsb->isb", Lf, X).reshape(-1, X.shape[2])
    pos = {t: q for q, t in enumerate(Iprev)}
    rows = [pos[t[:-1]] * d + t[-1] for t in Inew]  # KeyError if nesting is violated
    return Lp[rows, :]


def rightframe(X, Rf, Jnext, Jnew):
    """Algorithm 5 (right): R'_{alpha,(s,j)} = X^s_{alpha,gamma} R_{gamma,j}, then keep columns Jnew."""
    Rp = np.einsum("asg,gj->asj", X, Rf).reshape(X.shape[0], -1)
    pos = {t: q for q, t in enumerate(Jnext)}
    cols = [t[0] * len(Jnext) + pos[t[1:]] for t in Jnew]
    return Rp[:, cols]


def pi_tensor(Lf, X1, X2, Rf):
    """Eq. (pifromframes): Pi[alpha, s, s', beta] = L X_l X_{l+1} R, as (L X_l)(X_{l+1} R)."""
    r1 = X1.shape[2]
    LX = (Lf @ X1.reshape(X1.shape[0], -1)).reshape(-1, r1)
    XR = X2.reshape(-1, X2.shape[2]) @ Rf
    XR = XR.reshape(r1, -1)
    return (LX @ XR).reshape(Lf.shape[0], X1.shape[1], X2.shape[1], Rf.shape[1])


# ---------------------------------------------------------------- Algorithm 1: ACI

def init_guess(inputs, chimax: int, seed: int, complex_values: bool):
    """R9: counter-based random TT with bonds min(chi_hat, min_n r^n_s, prod_{t<s} d_t, prod_{t>=s} d_t)."""
    L = len(inputs[0])
    dims = [c.shape[1] for c in inputs[0]]
    ranks = [1]
    for s in range(1, L):
        full = min(int(np.prod(dims[:s], dtype=float)), int(np.prod(dims[s:], dtype=float)))
        ranks.append(min([chimax, full] + [int(x[s].shape[0]) for x in inputs]))
    ranks.append(1)
    return random_tt_counter(seed, ranks, dims, complex_values)


def _maxabs(a) -> float:
    return float(magnitude(a).max()) if a.size else 0.0


def assemble_output(factors, L: int):
    """R6: Y_0 = A_0, Y_s = B_{s-1} P_s^-1 (1 <= s <= L-2), Y_{L-1} = B_{L-2}."""
    Y = [None] * L
    if L == 1:
        return [factors["single"]]
    f0 = factors[0]
    Y[0] = f0["A"].reshape(1, -1, f0["k"])
    for s in range(1, L):
        B = factors[s - 1]["B"]  # k_{s-1} x (d_s * k_s)
        kprev = B.shape[0]
        if s == L - 1:
            Y[s] = B.reshape(kprev, -1, 1)
            continue
        fs = factors[s]
        k = fs["k"]
        X = B.reshape(-1, k)  # rows (alpha, sigma_s), columns J_{s+1}
        LI = fs["L"][fs["I"], :]
        UJ = fs["U"][:, fs["J"]]
        # X P^-1 with P = LI D UJ:  W UJ = X,  Z LI = W D^-1
        W = solve_triangular(UJ.T, X.T, lower=True, unit_diagonal=True).T
        W = W * _inv_diag(fs["D"])[None, :]
        Z = solve_triangular(LI.T, W.T, lower=False, unit_diagonal=True).T
        Y[s] = Z.reshape(kprev, -1, k)
    return Y


def aci(inputs, op: str = "mul", tol: float = 1e-10, max_rank: int = 64, *,
        tol_kind: str = "rel", maxiter: int = 20, coef=None, init=None, seed: int = 0,
        record: bool = False, pivot_mode: str = "full", follow=None, follow_slack: float = 1e-12,
        on_iteration=None):
    """Algorithm 1: alternating cross interpolation of f(X^1, ..., X^N).

    ``inputs`` is a list of N TTs (lists of cores (r, d, r')). Returns a dict with the
    output cores ``Y``, the ranks, the final pivot positions per bond (``I_pos``,
    ``J_pos``: row / column positions in that bond's Pi matrix, from the last sweep),
    ``eps`` per bond (last iteration, both half-sweeps), ``iterations``, ``S``, the pivots
    of every local update (``history``: {(u, b): (rows, cols)} with u = 0 for the initial
    CI, whose update of site s is filed under bond s - 1, and u = 1 + 2 (i - 1) + h for
    half-sweep h = 0 (left to right) / 1 (right to left) of iteration i) and, if ``record``,
    the per-pivot magnitudes needed to detect near-ties.

    ``follow``: a history in that format from another implementation. Every local update
    then takes the other side's pivots wherever they are as valid as its own (see ldu: within
    ``follow_slack`` times the scale of the matrix, S or max|M| for the initial CI), and the
    result's ``follow`` entry counts the updates and pivots compared, the steps where the two
    choices differed (near-ties) and lists every breach. Full search only.

    ``on_iteration(i)``, if given, is called after iteration i (both half-sweeps and the stop
    test) with no effect on the computation (used to time the oracle sweep by sweep).
    """
    N = len(inputs)
    L = len(inputs[0])
    dims = [c.shape[1] for c in inputs[0]]
    for x in inputs:
        assert len(x) == L and [c.shape[1] for c in x] == dims
    cplx = any(np.iscomplexobj(c) for x in inputs for c in x)
    if coef is not None and np.iscomplexobj(np.asarray(coef)):
        cplx = True
    dt = np.complex128 if cplx else np.float64
    X = [[np.asarray(c, dtype=dt) for c in x] for x in inputs]
    chimax = int(max_rank)
    rel = tol_kind == "rel"

    def fvals(blocks):
        return apply_op(op, blocks, coef)

    if L == 1:
        y = fvals([x[0] for x in X]).astype(dt)
        return dict(Y=[y], ranks=[1, 1], iterations=0, eps=[], I_pos=[], J_pos=[], S=_maxabs(y))

    Yinit = init if init is not None else init_guess(X, chimax, seed, cplx)
    Y = [np.asarray(c, dtype=dt).copy() for c in Yinit]

    # index sets: I[s] over sites 0..s, J[s] over sites s..L-1; I[-1] = J[L] = [()]
    I = {-1: [()]}
    J = {L: [()]}
    Lf = [{-1: np.ones((1, 1), dtype=dt)} for _ in range(N)]
    Rf = [{L: np.ones((1, 1), dtype=dt)} for _ in range(N)]

    history = {}
    freport = dict(updates=0, pivots=0, differ=0, violations=[])

    def followed(u, b, f):
        history[(u, b)] = (np.asarray(f["I"]).copy(), np.asarray(f["J"]).copy())
        if follow is not None:
            freport["updates"] += 1
            freport["pivots"] += f["k"]
            freport["differ"] += f["differ"]
            freport["violations"] += [(u, b) + v for v in f["violations"]]

    def fol(u, b):
        if follow is None:
            return None
        if (u, b) not in follow:
            raise ValueError(f"the followed history has no update {(u, b)}")
        return follow[(u, b)]

    # ---- CI-canonicalisation of the initial guess, right to left (R7)
    for s in range(L - 1, 0, -1):
        r = Y[s].shape[0]
        M = Y[s].reshape(r, -1)
        tau0 = tol * _maxabs(M) if rel else tol
        f = crossinterpolate(M, tau0, chimax, "right", pivot_mode, fol(0, s - 1), follow_slack * _maxabs(M))
        followed(0, s - 1, f)
        nj = len(J[s + 1])
        J[s] = [(int(q) // nj,) + J[s + 1][int(q) % nj] for q in f["J"]]
        Y[s] = f["B"].reshape(f["k"], dims[s], nj)
        Y[s - 1] = np.tensordot(Y[s - 1], f["A"], axes=(2, 0))
        for n in range(N):
            Rf[n][s] = rightframe(X[n][s], Rf[n][s + 1], J[s + 1], J[s])

    S = 0.0
    ranks_prev = [len(J[s]) for s in range(1, L)]
    J_prev = {s: list(J[s]) for s in range(1, L)}
    iterations = 0
    eps_lr = [0.0] * (L - 1)
    eps_rl = [0.0] * (L - 1)
    factors = {}
    I_pos = [None] * (L - 1)
    J_pos = [None] * (L - 1)
    log = []

    def bond(b, direction):
        nonlocal S
        blocks = [pi_tensor(Lf[n][b - 1], X[n][b], X[n][b + 1], Rf[n][b + 2]) for n in range(N)]
        Pi = fvals(blocks).astype(dt)
        S = max(S, _maxabs(Pi))
        tau = tol * S if rel else tol
        u = 1 + 2 * (iterations - 1) + (0 if direction == "right" else 1)
        f = localupdate(Pi, tau, chimax, direction, pivot_mode, fol(u, b), follow_slack * S)
        followed(u, b, f)
        ni = len(I[b - 1])
        nj = len(J[b + 2])
        I[b] = [I[b - 1][int(q) // dims[b]] + (int(q) % dims[b],) for q in f["I"]]
        J[b + 1] = [(int(q) // nj,) + J[b + 2][int(q) % nj] for q in f["J"]]
        Y[b] = f["Y"]
        Y[b + 1] = f["Y2"]
        if record:
            log.append(dict(bond=b, direction=direction, S=S, tau=tau, k=f["k"], eps=f["eps"],
                            best=f["best"], second=f["second"], I=f["I"].copy(), J=f["J"].copy()))
        return f

    for it in range(1, maxiter + 1):
        iterations = it
        for b in range(0, L - 1):  # left-to-right sweep
            f = bond(b, "right")
            eps_lr[b] = f["eps"]
            for n in range(N):
                Lf[n][b] = leftframe(X[n][b], Lf[n][b - 1], I[b - 1], I[b])
        for b in range(L - 2, -1, -1):  # right-to-left sweep
            f = bond(b, "left")
            eps_rl[b] = f["eps"]
            factors[b] = f
            I_pos[b] = f["I"].copy()
            J_pos[b] = f["J"].copy()
            for n in range(N):
                Rf[n][b + 1] = rightframe(X[n][b + 1], Rf[n][b + 2], J[b + 2], J[b + 1])
        ranks = [len(J[s]) for s in range(1, L)]
        tau = tol * S if rel else tol
        emax = max(max(eps_lr), max(eps_rl))
        grew = any(r > q for r, q in zip(ranks, ranks_prev))
        fixed = all(J[s] == J_prev[s] for s in range(1, L))
        if on_iteration is not None:
            on_iteration(it)
        if (not grew and emax <= tau) or fixed:
            break
        ranks_prev = ranks
        J_prev = {s: list(J[s]) for s in range(1, L)}

    Yout = assemble_output(factors, L)
    out = dict(Y=Yout, ranks=[1] + [len(J[s]) for s in range(1, L)] + [1], iterations=iterations,
               eps=[max(a, b) for a, b in zip(eps_lr, eps_rl)], eps_lr=list(eps_lr),
               eps_rl=list(eps_rl), I_pos=I_pos, J_pos=J_pos, S=S,
               I_sets={s: list(I[s]) for s in range(0, L - 1)},
               J_sets={s: list(J[s]) for s in range(1, L)}, history=history)
    if follow is not None:
        out["follow"] = freport
    if record:
        out["log"] = log
    return out
