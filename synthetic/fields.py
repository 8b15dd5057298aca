"""Seeded Fourier-field, Gaussian and random-TT inputs in quantics form.

Quantics grid (Eq. (quanticsrep)): x = sum_{l>=1} 2^-l sigma_l, site 0 holds the most
significant bit. 2D fields interleave the bits (x_1, y_1, x_2, y_2, ...); 3D fields fuse
one bit of each axis into a d=8 site, sigma = 4 b_x + 2 b_y + b_z.

A single Fourier mode exp(i theta(x)) with theta linear in x factorises over the bits,
so it is an exact rank-1 complex TT; its real part cos(theta + phi) is an exact rank-2
real TT built from 2x2 rotations. A field is the block sum of its modes, compressed
with TT-SVD to the requested rank.
"""

from __future__ import annotations

import numpy as np

from .tt import tt_block_sum, tt_svd_round, tt_from_dense, tt_random_uniform


def _site_angles(kvec, L, ndim, layout, scale):
    """Per-site phase increment a_s(sigma) (array (L, d)) for wavevector ``kvec``.

    theta(x) = scale * k.x, and x's bits enter linearly, so theta = sum_s a_s(sigma_s).
    """
    if layout == "1d":
        d = 2
        ang = np.zeros((L, d))
        for s in range(L):
            ang[s, 1] = scale * kvec[0] * 0.5 ** (s + 1)
        return ang
    if layout == "interleaved":
        d = 2
        ang = np.zeros((L, d))
        for s in range(L):
            axis = s % ndim
            bit = s // ndim
            ang[s, 1] = scale * kvec[axis] * 0.5 ** (bit + 1)
        return ang
    if layout == "fused":
        d = 2 ** ndim
        ang = np.zeros((L, d))
        for s in range(L):
            for sig in range(d):
                tot = 0.0
                for axis in range(ndim):
                    b = (sig >> (ndim - 1 - axis)) & 1
                    tot += kvec[axis] * b
                ang[s, sig] = scale * tot * 0.5 ** (s + 1)
        return ang
    raise ValueError(layout)


def cos_mode_tt(amp, phase, ang):
    """Exact rank-2 real TT of amp * cos(phase + sum_s ang[s, sigma_s])."""
    L, d = ang.shape
    cores = []
    for s in range(L):
        a = ang[s]
        c, sn = np.cos(a), np.sin(a)
        if s == 0:
            core = np.zeros((1, d, 2))
            core[0, :, 0] = amp * np.cos(phase + a)
            core[0, :, 1] = amp * np.sin(phase + a)
            if L == 1:
                core = core[:, :, :1]
        elif s == L - 1:
            core = np.zeros((2, d, 1))
            core[0, :, 0] = c
            core[1, :, 0] = -sn
        else:
            core = np.zeros((2, d, 2))
            core[0, :, 0] = c
            core[0, :, 1] = sn
            core[1, :, 0] = -sn
            core[1, :, 1] = c
        cores.append(core)
    return cores


def exp_mode_tt(amp, ang):
    """Exact rank-1 complex TT of amp * exp(i sum_s ang[s, sigma_s])."""
    L, d = ang.shape
    cores = []
    for s in range(L):
        core = np.exp(1j * ang[s]).reshape(1, d, 1).astype(np.complex128)
        if s == 0:
            core = core * amp
        cores.append(core)
    return cores


def _disc_lattice(ndim, kmax):
    rng1 = np.arange(-kmax, kmax + 1)
    grids = np.meshgrid(*([rng1] * ndim), indexing="ij")
    pts = np.stack([g.reshape(-1) for g in grids], axis=1)
    keep = (pts ** 2).sum(axis=1) <= kmax * kmax
    return pts[keep]


def fourier_config1(seed: int):
    """1D, L=12, d=2: Re sum_{k=-8..8} c_k e^{2 pi i k x}, c_k ~ N(0,1) exp(-k^2/16), TT-SVD rel 1e-12."""
    rng = np.random.default_rng(seed)
    L = 12
    ks = np.arange(-8, 9)
    ck = rng.standard_normal(len(ks)) * np.exp(-ks.astype(float) ** 2 / 16.0)
    modes = [cos_mode_tt(ck[i], 0.0, _site_angles([k], L, 1, "1d", 2 * np.pi)) for i, k in enumerate(ks)]
    return tt_svd_round(tt_block_sum(modes), rel_tol=1e-12), dict(ks=ks, ck=ck)


def fourier_config2(seed: int, chi: int, nbits: int = 20, nmodes: int = 200, kmax: int = 32):
    """2D interleaved, L=2*nbits, d=2: sum_k a_k cos(2 pi k.x + phi_k), TT-SVD to rank chi.

    ``nmodes`` distinct k with |k| <= kmax drawn without replacement from the disc lattice;
    a_k ~ N(0,1) exp(-|k|^2/100), phi_k ~ U[0, 2 pi).
    """
    rng = np.random.default_rng(seed)
    L = 2 * nbits
    lat = _disc_lattice(2, kmax)
    idx = rng.choice(len(lat), size=nmodes, replace=False)
    kv = lat[idx]
    amp = rng.standard_normal(nmodes) * np.exp(-(kv.astype(float) ** 2).sum(axis=1) / 100.0)
    phase = rng.uniform(0.0, 2 * np.pi, size=nmodes)
    modes = [cos_mode_tt(amp[i], phase[i], _site_angles(kv[i], L, 2, "interleaved", 2 * np.pi))
             for i in range(nmodes)]
    cores = tt_svd_round(tt_block_sum(modes), max_rank=chi)
    return cores, dict(k=kv, amp=amp, phase=phase)


def fourier_config3(seed: int, chi: int, nsites: int = 12, nmodes: int = 500, kmax: int = 24):
    """3D fused d=8, ``nsites`` sites: sum_k a_k exp(2 pi i k.x), a_k ~ (N + iN)/sqrt2 exp(-|k|^2/100)."""
    rng = np.random.default_rng(seed)
    lat = _disc_lattice(3, kmax)
    idx = rng.choice(len(lat), size=nmodes, replace=False)
    kv = lat[idx]
    amp = (rng.standard_normal(nmodes) + 1j * rng.standard_normal(nmodes)) / np.sqrt(2.0)
    amp = amp * np.exp(-(kv.astype(float) ** 2).sum(axis=1) / 100.0)
    modes = [exp_mode_tt(amp[i], _site_angles(kv[i], nsites, 3, "fused", 2 * np.pi)) for i in range(nmodes)]
    cores = tt_svd_round(tt_block_sum(modes), max_rank=chi)
    return cores, dict(k=kv, amp=amp)


def fourier_paper_1d(seed: int, K: int, L: int = 30, rel_tol: float = 1e-12):
    """Sec. 3.2, Eq. (fourierseries): g(x) = sum_{k=0}^K g_k e^{ikx} on [0,1), Re/Im g_k ~ U[0,1],
    normalised so sum |g_k|^2 = 1."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(0, 1, K + 1) + 1j * rng.uniform(0, 1, K + 1)
    g = g / np.sqrt((np.abs(g) ** 2).sum())
    modes = [exp_mode_tt(g[k], _site_angles([k], L, 1, "1d", 1.0)) for k in range(K + 1)]
    cores = tt_svd_round(tt_block_sum(modes), rel_tol=rel_tol)
    return cores, dict(g=g)


def fourier_paper_1d_large(seed: int, K: int, L: int = 30, chunk: int = 256, rel_tol: float = 1e-12):
    """fourier_paper_1d for large K: the same coefficients; the modes are summed in chunks of
    ``chunk`` consecutive frequencies (each chunk a block sum rounded by TT-SVD), and the chunks
    are then added pairwise with TT-SVD rounding after every sum, so no block sum is wider than
    twice the series' own rank."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(0, 1, K + 1) + 1j * rng.uniform(0, 1, K + 1)
    g = g / np.sqrt((np.abs(g) ** 2).sum())
    parts = []
    for k0 in range(0, K + 1, chunk):
        modes = [exp_mode_tt(g[k], _site_angles([k], L, 1, "1d", 1.0)) for k in range(k0, min(K + 1, k0 + chunk))]
        parts.append(tt_svd_round(tt_block_sum(modes), rel_tol=rel_tol))
    while len(parts) > 1:
        nxt = [tt_svd_round(tt_block_sum(parts[i:i + 2]), rel_tol=rel_tol) if i + 1 < len(parts) else parts[i]
               for i in range(0, len(parts), 2)]
        parts = nxt
    return parts[0], dict(g=g)


def gaussian_pair(L: int, w: float, delta: float, rel_tol: float = 1e-15):
    """Sec. 3.1, Eq. (gaussians): g_pm(x) = exp(-(x pm delta/2)^2 / (2 w^2)) on x in [-0.5, 0.5),
    as TT-SVD of the dense 2^L-point vectors."""
    x = -0.5 + np.arange(2 ** L) / 2.0 ** L
    gp = np.exp(-(x + delta / 2) ** 2 / (2 * w * w))
    gm = np.exp(-(x - delta / 2) ** 2 / (2 * w * w))
    dims = [2] * L
    return tt_from_dense(gp, dims, rel_tol=rel_tol), tt_from_dense(gm, dims, rel_tol=rel_tol), x


def random_tt_pair(seed: int, L: int, d: int, chi: int, dtype=np.float64):
    """Sec. 3.3: two TTs with uniform random cores."""
    rng = np.random.default_rng(seed)
    return (tt_random_uniform(rng, L, d, chi, dtype=dtype),
            tt_random_uniform(rng, L, d, chi, dtype=dtype))


CONFIG_NAMES = {
    1: "1D quantics L=12 d=2 FP64, Fourier sums k=-8..8, op a*b, tol 1e-10",
    2: "2D interleaved quantics L=40 d=2 FP64, 200-mode Fourier fields, op a*b, tol 1e-10",
    3: "3D quantics 12 sites d=8 complex128, 500-mode field, op |psi|^2 psi, tol 1e-8",
}


def sequence_config5_pair(t: int, chi: int, nbits: int = 20, nmodes: int = 200, kmax: int = 32, seed: int = 1005):
    """Step t of the learned-proposal sequence: f_t and g_t are 2D interleaved Fourier fields as in
    config 2 whose every mode's phase advances by omega_k t, omega_k ~ U[0, 1] (the modes, amplitudes,
    initial phases and omegas fixed by ``seed``); TT-SVD to rank chi."""
    out = []
    for which in (0, 1):
        rng = np.random.default_rng(seed * 10 + which)
        L = 2 * nbits
        lat = _disc_lattice(2, kmax)
        idx = rng.choice(len(lat), size=nmodes, replace=False)
        kv = lat[idx]
        amp = rng.standard_normal(nmodes) * np.exp(-(kv.astype(float) ** 2).sum(axis=1) / 100.0)
        phase0 = rng.uniform(0.0, 2 * np.pi, size=nmodes)
        omega = rng.uniform(0.0, 1.0, size=nmodes)
        phase = phase0 + omega * t
        modes = [cos_mode_tt(amp[i], phase[i], _site_angles(kv[i], L, 2, "interleaved", 2 * np.pi))
                 for i in range(nmodes)]
        out.append(tt_svd_round(tt_block_sum(modes), max_rank=chi))
    return out[0], out[1]


def batch_config4_spec(seed: int = 1004, n: int = 64):
    """The batched workload: n independent pairs of 2D interleaved Fourier fields as in config 2,
    with lengths L = 2 * nbits, nbits uniform in [10, 20] (L uniform over the even values in
    [20, 40]), ranks chi uniform in [16, 256], 200 modes per field as in config 2 (TT-SVD
    truncates each to rank chi), ops alternating a*b and a*conj(b) (the same for real fields),
    even pairs FP64 and odd pairs FP32 (``dtype``: the element type the pair is handed over in).
    The configuration fixes neither tolerance nor rank cap: tol 1e-8 (relative) and max_rank chi.
    Returns the per-pair parameters; ``batch_config4_pair`` builds one pair (in FP64)."""
    rng = np.random.default_rng(seed)
    spec = []
    for i in range(n):
        nbits = int(rng.integers(10, 21))
        chi = int(rng.integers(16, 257))
        spec.append(dict(index=i, nbits=nbits, chi=chi, nmodes=200,
                         op="mul" if i % 2 == 0 else "mul_conj", tol=1e-8, max_rank=chi,
                         dtype="f64" if i % 2 == 0 else "f32",
                         seed_a=seed * 1000 + 2 * i, seed_b=seed * 1000 + 2 * i + 1))
    return spec


def batch_config4_pair(spec: dict):
    a, _ = fourier_config2(spec["seed_a"], spec["chi"], nbits=spec["nbits"], nmodes=spec["nmodes"])
    b, _ = fourier_config2(spec["seed_b"], spec["chi"], nbits=spec["nbits"], nmodes=spec["nmodes"])
    return a, b


def config_inputs(cfg: int, chi: int | None = None):
    """Inputs and call parameters for a workload; seeds A = 1000 + cfg, B = 2000 + cfg."""
    if cfg == 1:
        a, _ = fourier_config1(1001)
        b, _ = fourier_config1(2001)
        return dict(inputs=[a, b], op="mul", tol=1e-10, max_rank=64)
    if cfg == 2:
        chi = 128 if chi is None else chi
        a, _ = fourier_config2(1002, chi)
        b, _ = fourier_config2(2002, chi)
        return dict(inputs=[a, b], op="mul", tol=1e-10, max_rank=2 * chi)
    if cfg == 3:
        chi = 128 if chi is None else chi
        a, _ = fourier_config3(1003, chi)
        return dict(inputs=[a], op="abs2_mul", tol=1e-8, max_rank=chi)
    raise ValueError(f"unknown config {cfg}")
