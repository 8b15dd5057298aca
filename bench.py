#!/usr/bin/env python
"""Benchmark of one ACI product f(A, B) = A * B on GB300 (replicas across GPUs).

Workload (default): 2D interleaved quantics TTs, L = 40 sites (2 x 20 bits), d = 2, FP64 real,
seeded 200-mode Fourier fields (|k| <= 32, amplitudes N(0,1) exp(-|k|^2/100)) as exact block
sums, TT-SVD to rank chi = 128; op a*b, tol 1e-10 relative, max_rank 2 chi = 256, at most 20
sweeps. One step = one whole ACI call (initial guess, sweeps, stop tests, output assembly)
through the C ABI on device-resident inputs.

Prints one JSON line (rank 0). `value` = products per second over all ranks. The L2 cache is
flushed (a 256 MB write, outside the timed events) before every timed step. The `roofline`
object is for the kernel class with the largest share of device time, from CUDA events recorded
by the library on its stream around every launch during the timed steps. `cpu_baseline` times
the CPU oracle on a bounded sample of the same workload on this host. `mixed` repeats the
workload with the frame and Pi contractions on the tensor cores (BF16 digit planes, --mixed-digits
of them) and states its sampled error against the exact product and against the FP64 result, with
a tensor-pipe roofline for those contractions.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ACI f(A,B) time vs χ at rel err ≤1e-8 (FP64 vs mixed/learned); % tensor peak"
UNIT = "products/s"
# FP64 vector peak of a GB300, nominal 1.25 TFLOP/s (152 SMs x ~2 DFMA/clk/SM at ~2.06 GHz); the
# rooflines use the library's own FP64 probe (aci_k_fp64_peak) measured in the same run instead.
FP64_NOMINAL_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--chi", type=int, default=128)
    ap.add_argument("--max-sweeps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-threads", type=int, default=1,
                    help="reference arm: BLAS threads of the oracle (0: the library default); one thread is the "
                         "faster on its matrices of at most a few hundred rows")
    ap.add_argument("--no-time-to-tol", dest="time_to_tol", action="store_false",
                    help="skip the per-sweep time and error curve")
    ap.add_argument("--no-cfg3", dest="cfg3", action="store_false", help="skip the fused d = 8 sub-object")
    ap.add_argument("--cfg3-chi", type=int, default=128)
    ap.add_argument("--vs-chi", default="32,64,96", help="other input ranks of the workload timed beside the "
                                                        "headline (empty: skip)")
    ap.add_argument("--batch-line", type=int, default=64,
                    help="pairs of the batched workload in the default line's batch object (0: skip it)")
    ap.add_argument("--mixed-digits", type=int, default=6, help="BF16 digit planes of the mixed run (0: skip it)")
    ap.add_argument("--precision", default="fp64", help="contractions of the headline run: fp64 or bf16xS")
    ap.add_argument("--pivot-mode", default="full", choices=["full", "rook"])
    ap.add_argument("--autotune", type=int, default=1,
                    help="1 (default): the contraction tuner (aci_opts.autotune) for the headline run; 0: off")
    ap.add_argument("--overlap", default="auto", choices=["auto", "off", "on"],
                    help="schedule of the sweeps (aci_opts.sweep_overlap)")
    ap.add_argument("--kernel", default="", choices=["", "pi_block", "frame_gemm", "prrlu", "fp64peak"],
                    help="time one step-level call of this shape instead of the product (kernel profiling)")
    ap.add_argument("--m", type=int, default=2048)
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--k", type=int, default=256)
    ap.add_argument("--complex", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="time this many independent pairs of the batched workload instead (aci_elementwise_batch)")
    ap.add_argument("--streams", type=int, default=0, help="batch: products in flight (0 = library default)")
    ap.add_argument("--proposer-line", type=int, default=9,
                    help="steps of the learned-proposal sequence (chi 128) in the default line's proposer object "
                         "(0: skip it)")
    ap.add_argument("--proposer", action="store_true",
                    help="the learned-proposal sequence: train on steps 0-39, compare on 40-59")
    ap.add_argument("--seq-steps", type=int, default=60)
    ap.add_argument("--scaling", action="store_true", help="time vs chi on the paper's scaling workloads")
    ap.add_argument("--scaling-fourier", default="64,256,1024,4096,16384,32768", help="K values (Sec. 3.2)")
    ap.add_argument("--scaling-random", default="8,16,32,64,128,256", help="chi values (Sec. 3.3)")
    ap.add_argument("--scaling-sweeps", type=int, default=2, help="sweeps of the random-TT products (tol 0)")
    ap.add_argument("--scaling-cpu-chi", type=int, default=256, help="largest input chi the CPU oracle's ACI runs")
    ap.add_argument("--scaling-kron-chi", type=int, default=32, help="largest input chi of the CPU Kronecker product")
    ap.add_argument("--keep", default="1.25",
                    help="proposer: kept candidates per side = keep x previous rank + 8; a comma list compares several")
    return ap.parse_args()


def _seq_pair(args):
    t, chi = args
    from synthetic.fields import sequence_config5_pair
    return sequence_config5_pair(t, chi)


def make_sequence(nsteps, chi):
    """The learned-proposal sequence's inputs, generated in a spawned pool (before any GPU call)."""
    import multiprocessing as mp
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        pairs = pool.map(_seq_pair, [(t, chi) for t in range(nsteps)])
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.pop(v, None)
    return pairs, time.time() - t0


def proposer_measure(ctx, pairs, chi, keeps, max_sweeps, gen_s):
    """Plain ACI runs the first two thirds of the sequence while recording the (features, pivot-or-
    not) pairs of its left-to-right updates; the network is trained on them with the library's
    kernels (Adam, weighted logistic loss); the remaining steps run with plain ACI and with the
    learned restriction. Returns the time per product and the error against the exact product on
    20000 sampled points of each, and the held-out AUC of the scores."""
    import numpy as np
    import torch
    from synthetic.tt import tt_eval
    from synthetic.weights import proposer_init
    nsteps = len(pairs)
    ntrain = (2 * nsteps) // 3
    tol, max_rank = 1e-8, 2 * chi
    dev = lambda tt: [torch.from_numpy(c).cuda() for c in tt]
    read = ctx.record_proposer_data(4_000_000)
    for t in range(ntrain):
        a, b = pairs[t]
        ctx.elementwise(dev(a), dev(b), "mul", tol, max_rank, max_sweeps=max_sweeps)
    X, y, nrec = read()
    pos = float(y.mean().item())
    P = torch.from_numpy(proposer_init(0, 7)).cuda()
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    t1 = time.time()
    for it in range(1, 401):
        loss, g = ctx.mlp_grad(X, y, P, (1 - pos) / max(pos, 1e-6))
        ctx.mlp_adam(P, g, M, V, it, 2e-3)
    torch.cuda.synchronize()
    train_s = time.time() - t1
    print(f"proposer: {X.shape[0]} records ({pos:.3f} positive), loss {loss:.4f}, {train_s:.1f} s", file=sys.stderr,
          flush=True)
    rng = np.random.default_rng(8)
    modes = ["plain"] + ["proposed" if i == 0 else f"proposed@{k:g}" for i, k in enumerate(keeps)]
    rows = {m: [] for m in modes}
    for t in range(ntrain, nsteps):
        a, b = pairs[t]
        pts = rng.integers(0, 2, size=(20000, len(a)))
        exact = tt_eval(a, pts) * tt_eval(b, pts)
        A, B = dev(a), dev(b)
        for mi, mode in enumerate(modes):
            if mode != "plain":
                ctx.set_proposer(P, keep=keeps[mi - 1])
            for rep in range(2):  # the second run is timed
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ycores, info = ctx.elementwise(A, B, "mul", tol, max_rank, max_sweeps=max_sweeps,
                                               pivot_mode="full" if mode == "plain" else "proposed")
                e1.record()
                torch.cuda.synchronize()
            yv = tt_eval([c.cpu().numpy() for c in ycores], pts)
            rows[mode].append((e0.elapsed_time(e1), float(np.abs(yv - exact).max() / np.abs(exact).max()),
                               info["iterations"], max(info["ranks"])))
            ctx.set_proposer(None)
    summ = {m: {"ms_per_product": float(np.mean([r[0] for r in v])),
                "max_rel_err_vs_exact": float(np.max([r[1] for r in v])),
                "mean_iterations": float(np.mean([r[2] for r in v])),
                "max_rank": int(np.max([r[3] for r in v]))} for m, v in rows.items()}
    # held-out AUC of the scores on a recorded held-out product
    read = ctx.record_proposer_data(2_000_000)
    a, b = pairs[nsteps - 1]
    ctx.elementwise(dev(a), dev(b), "mul", tol, max_rank, max_sweeps=max_sweeps)
    Xt, yt, _ = read()
    zt = ctx.mlp_forward(Xt, P, fp16=True).cpu().numpy()
    yt = yt.cpu().numpy()
    sub = np.random.default_rng(9)
    zp, zn = zt[yt > 0.5], zt[yt < 0.5]
    zp = zp[sub.permutation(len(zp))[:2000]]
    zn = zn[sub.permutation(len(zn))[:2000]]
    return {"workload": f"{nsteps}-step sequence f_t g_t of 2D interleaved Fourier fields (L=40, d=2, chi={chi}), "
                        f"phases advancing by omega_k t; tol {tol:g}, max_rank {max_rank}; trained on steps "
                        f"0-{ntrain - 1}, compared on {ntrain}-{nsteps - 1}",
            "keep": keeps, "input_generation_s": gen_s,
            "training": {"records": int(X.shape[0]), "positive_share": pos, "final_loss": loss,
                         "adam_steps": 400, "train_s": train_s},
            **{m: summ[m] for m in modes},
            "speedup": summ["plain"]["ms_per_product"] / summ["proposed"]["ms_per_product"],
            **{f"speedup@{k:g}": summ["plain"]["ms_per_product"] / summ[m]["ms_per_product"]
               for k, m in zip(keeps, modes[1:])},
            "held_out_auc": float((zp[:, None] > zn[None, :]).mean()) if len(zp) and len(zn) else float("nan")}


def run_proposer(args):
    """The learned-proposal sequence alone (bench.py --proposer): see proposer_measure."""
    pairs, gen_s = make_sequence(args.seq_steps, args.chi)
    print(f"proposer: {len(pairs)} steps generated in {gen_s:.1f} s", file=sys.stderr, flush=True)
    from paper_2604_00037_gb300.binding import Context
    ctx = Context(0)
    keeps = [float(k) for k in str(args.keep).split(",")]
    res = proposer_measure(ctx, pairs, args.chi, keeps, args.max_sweeps, gen_s)
    line = {"metric": "learned pivot proposal: ACI time per product at equal error (held-out steps)",
            "unit": "ms/product", "value": res["proposed"]["ms_per_product"], "higher_is_better": False,
            "dtype": "f64", "data": "synthetic", "n_gpus": 1, "config": {"workload": res["workload"]}, **res}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_batch(args):
    """The batched workload alone: args.batch pairs (synthetic/fields.py, batch_config4_spec) through
    aci_elementwise_batch, one product at a time and concurrently (autotuned), device-resident inputs."""
    spec, pairs, gen_s = make_batch(args.batch)
    print(f"batch: {len(pairs)} pairs generated in {gen_s:.1f} s", file=sys.stderr, flush=True)
    import torch
    from paper_2604_00037_gb300.binding import Context
    ctx = Context(0)
    line = run_batch_line(ctx, spec, pairs, gen_s, args, torch.cuda.current_stream(), reps=max(1, args.steps))
    line = {"metric": "batched ACI products/s (independent pairs of uneven L and chi)", "higher_is_better": True,
            "dtype": "f64 (odd pairs handed over in FP32)", "data": "synthetic", "n_gpus": 1, "steps": args.steps,
            **line}
    print(json.dumps(line), flush=True)
    ctx.close()


def _scaling_input(job):
    """One input of the scaling workloads (in a worker process): ("fourier", seed, K) or
    ("random", seed, chi)."""
    kind, seed, x = job
    if kind == "fourier":
        from synthetic.fields import fourier_paper_1d_large
        return fourier_paper_1d_large(seed, x)[0]
    import numpy as np
    from synthetic.tt import tt_random_uniform
    return tt_random_uniform(np.random.default_rng(seed), 30, 2, x)


def _oracle_time(job):
    """Wall time of one CPU product (in a one-thread worker): ("aci" | "kron", a, b, tol, max_rank, sweeps)."""
    kind, a, b, tol, max_rank, sweeps = job
    t0 = time.perf_counter()
    if kind == "aci":
        import oracle
        oracle.aci([a, b], "mul", tol, max_rank, maxiter=sweeps, tol_kind="abs" if tol > 0 else "rel")
    else:
        from oracle.hadamard import hadamard_kron, tt_round_svd
        tt_round_svd(hadamard_kron(a, b), max_rank=max_rank, rel_tol=tol)
    return time.perf_counter() - t0


def _fit(xs, ts):
    import numpy as np
    if len(xs) < 2:
        return None
    p, c = np.polyfit(np.log(np.asarray(xs, float)), np.log(np.asarray(ts, float)), 1)
    return float(p)


def run_scaling(args):
    """Time vs chi on the paper's scaling workloads, FP64 / complex128 on one GPU, with fitted
    power laws t ~ chi^p (Sec. 3.2: products of two random Fourier series, 1D quantics L = 30,
    tol 1e-8, the ranks set by the tolerance; Sec. 3.3: products of uniform random TTs, L = 30,
    d = 2, output rank capped at chi' = chi). Beside them, on one CPU thread each, the oracle's
    ACI and the O(chi^4) Kronecker-delta product with SVD rounding where they finish in seconds."""
    import multiprocessing as mp
    import numpy as np
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    Ks = [int(k) for k in args.scaling_fourier.split(",") if k]
    chis = [int(c) for c in args.scaling_random.split(",") if c]
    jobs = [("fourier", s, K) for K in Ks for s in (3001, 3002)] + [("random", s, c) for c in chis for s in (3003, 3004)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:  # before any GPU call
        made = pool.map(_scaling_input, jobs)
        inputs = {(j[0], j[2]): [] for j in jobs}
        for j, tt in zip(jobs, made):
            inputs[(j[0], j[2])].append(tt)
        cpu_jobs, cpu_keys = [], []
        for (kind, x), (a, b) in inputs.items():
            chi = max(c.shape[2] for c in a)
            tol, mr, sw = (1e-8, 4096, args.max_sweeps) if kind == "fourier" else (0.0, x, args.scaling_sweeps)
            if chi <= args.scaling_cpu_chi and (kind == "random" or chi <= 64):
                cpu_jobs += [("aci", a, b, tol, mr, sw)]
                cpu_keys += [(kind, x, "aci")]
            if chi <= args.scaling_kron_chi:
                cpu_jobs += [("kron", a, b, tol, mr, sw)]
                cpu_keys += [(kind, x, "kron")]
        cpu_times = dict(zip(cpu_keys, pool.map(_oracle_time, cpu_jobs)))
    gen_s = time.time() - t0
    import torch
    from paper_2604_00037_gb300.binding import Context
    from synthetic.tt import tt_eval
    ctx = Context(0)
    stream = torch.cuda.current_stream()
    rows = {"fourier": [], "random": []}
    rng = np.random.default_rng(21)
    for (kind, x), (a, b) in inputs.items():
        A, B = [torch.from_numpy(c).cuda() for c in a], [torch.from_numpy(c).cuda() for c in b]
        tol, mr, sw = (1e-8, 4096, args.max_sweeps) if kind == "fourier" else (0.0, x, args.scaling_sweeps)
        # Sec. 3.2's tau is absolute (the paper's Alg. 1); the random-TT products run at a rank cap
        call = lambda: ctx.elementwise(A, B, "mul", tol, mr, max_sweeps=sw, tol_kind="abs" if tol > 0 else "rel")
        call()
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            y, info = call()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        pts = rng.integers(0, 2, size=(1000, len(a)))  # the paper samples 10^3 points
        exact = tt_eval(a, pts) * tt_eval(b, pts)
        diff = float(np.abs(tt_eval([c.cpu().numpy() for c in y], pts) - exact).max())
        chi = max(c.shape[2] for c in a)
        row = {"x": x, "chi": chi, "chi_out": max(info["ranks"]), "sweeps": info["iterations"],
               "gpu_ms": statistics.median(ts), "max_abs_err": diff, "max_rel_err": diff / float(np.abs(exact).max()),
               "oracle_aci_s": cpu_times.get((kind, x, "aci")), "oracle_kron_s": cpu_times.get((kind, x, "kron"))}
        rows[kind].append(row)
        print(json.dumps({kind: row}), file=sys.stderr, flush=True)
    fits = {}
    for kind, rr in rows.items():
        rr.sort(key=lambda r: r["chi"])

        def top3(key):  # the three largest chi timed in a column (smaller ones are overhead-bound)
            pts = [(r["chi"], r[key]) for r in rr if r[key]][-3:]
            return _fit([p[0] for p in pts], [p[1] for p in pts])
        fits[kind] = {"gpu": top3("gpu_ms"), "oracle_aci": top3("oracle_aci_s"), "oracle_kron": top3("oracle_kron_s")}
    line = {"metric": "ACI product time vs chi (paper's scaling workloads), fitted exponent p of t ~ chi^p",
            "unit": "ms/product", "dtype": "complex128 (Fourier) / f64 (random)", "data": "synthetic", "n_gpus": 1,
            "config": {"fourier": f"Sec. 3.2: two random Fourier series of K+1 modes, K in {Ks}, 1D quantics L = 30, "
                                  f"a*b, absolute tau 1e-8 as in the paper, <= {args.max_sweeps} sweeps",
                       "random": f"Sec. 3.3: uniform random TTs, L = 30, d = 2, chi in {chis}, chi' <= chi (tol 0), "
                                 f"{args.scaling_sweeps} sweeps",
                       "fit": "least squares on log t vs log chi over the three largest chi timed in each column",
                       "cpu": "one thread per product", "input_generation_s": gen_s},
            "fourier": rows["fourier"], "random": rows["random"], "exponents": fits,
            "paper_exponents": {"aci": 2.3, "kron": 3.8, "source": "Sec. 3.2, Fig. 2 (single CPU thread, context only)"}}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_kernel(args):
    """One step-level call, repeated: the Pi block f = |a|^2 a (m x n, K = k), a frame product
    (m x k times k x n) or the pivot search (m x n, k pivots) on seeded Gaussian inputs."""
    import numpy as np
    import torch
    from paper_2604_00037_gb300.binding import Context
    ctx = Context(0)
    rng = np.random.default_rng(0)

    def mat(r, c):
        x = rng.standard_normal((r, c))
        if args.complex:
            x = x + 1j * rng.standard_normal((r, c))
        return torch.from_numpy(x).cuda()
    if args.kernel == "fp64peak":
        t = [ctx.fp64_peak() for _ in range(max(1, args.steps))]
        print(json.dumps({"kernel": "fp64peak", "tflops": t, "median_tflops": statistics.median(t),
                          "note": "aci_k_fp64_peak: 8 CTAs of 512 threads per SM, 8 independent FP64 FMA "
                                  "chains per thread, CUDA events"}), flush=True)
        ctx.close()
        return
    if args.kernel == "pi_block":
        A, B = mat(args.m, args.k), mat(args.k, args.n)
        call = lambda: ctx.pi_block([A], [B], "abs2_mul", precision=args.precision)
        flops = (8.0 if args.complex else 2.0) * args.m * args.n * args.k
    elif args.kernel == "frame_gemm":
        A, B = mat(args.m, args.k), mat(args.k, args.n)
        call = lambda: ctx.frame_gemm(A, B, precision=args.precision)
        flops = (8.0 if args.complex else 2.0) * args.m * args.n * args.k
    else:
        r = min(args.m, args.n, 300)
        M = (mat(args.m, r) @ mat(r, args.n)).contiguous()
        call = lambda: ctx.prrlu(M, 0.0, args.k, mode=args.pivot_mode)
        flops = None
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    line = {"kernel": args.kernel, "m": args.m, "n": args.n, "k": args.k, "complex": args.complex,
            "precision": args.precision, "pivot_mode": args.pivot_mode, "ms_per_call": ms,
            "note": "per call including the host synchronisation of the step-level entry"}
    if flops:
        line["fp64_equivalent_tflops"] = flops / (ms / 1e3) / 1e12
    print(json.dumps(line), flush=True)
    ctx.close()


def measured_peak(key, fallback):
    """A peak from the measured MEASURED_PEAKS.json, else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def workload(chi):
    from synthetic import config_inputs
    p = config_inputs(2, chi)
    return p


def config_dict(args, p):
    return {"workload": f"2D interleaved quantics FP64 Fourier fields, L=40 d=2, chi={args.chi}, "
                        f"a*b, tol {p['tol']:g} rel, max_rank {p['max_rank']}, <= {args.max_sweeps} sweeps",
            "L": 40, "d": 2, "chi": args.chi, "max_rank": p["max_rank"], "tol": p["tol"],
            "op": "a*b", "max_sweeps": args.max_sweeps,
            "contractions": args.precision, "pivot_search": args.pivot_mode, "sweep_overlap": args.overlap,
            "contraction_tuner": bool(args.autotune),
            "l2": "flushed before every timed step (256 MB write, untimed)",
            "parallelism": f"replicas x{args.gpus}"}


# ------------------------------------------------------------------------------ CPU oracle

def oracle_product(p, max_sweeps, max_iters=None):
    """One oracle product of the workload, timed sweep by sweep (wall clock). Returns (total seconds,
    cumulative seconds after each sweep iteration, iterations run). ``max_iters`` stops it early."""
    import oracle
    a, b = p["inputs"]
    marks = []
    t0 = time.perf_counter()
    oracle.aci([a, b], "mul", p["tol"], p["max_rank"], maxiter=max_iters or max_sweeps,
               on_iteration=lambda it: marks.append(time.perf_counter() - t0))
    return time.perf_counter() - t0, marks, len(marks)


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info()]
        return max(n) if n else 1
    except Exception:
        env = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS")
        return int(env) if env else (os.cpu_count() or 1)


def oracle_subprocess(chi, max_sweeps, threads, iters=None):
    """One oracle product in a child process with `threads` BLAS threads (the count is fixed when
    numpy loads). Returns (seconds, sweeps) or None."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS=str(threads), OMP_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "p = bench.workload(%d); t, m, n = bench.oracle_product(p, %d, %s); print(json.dumps([t, n]))"
            % (ROOT, chi, max_sweeps, repr(iters)))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
        t, n = json.loads(r.stdout.strip().splitlines()[-1])
        return t, n
    except Exception:
        return None


def cpu_baseline_line(p, args):
    """The oracle timed on this host, one whole product each way: with every BLAS thread (in this
    process) and with one thread (a child process; the paper times one CPU thread). The value is
    the faster of the two (its matrices are at most a few hundred wide, where one thread can win)."""
    total, marks, iters = oracle_product(p, args.max_sweeps)
    allc = {"value": 1.0 / total, "cores": blas_threads(), "seconds_per_product": total, "sweeps": iters}
    one = oracle_subprocess(args.chi, args.max_sweeps, 1)
    out = {"unit": UNIT, "kind": "oracle", "all_threads": allc}
    best = allc
    if one:
        out["one_thread"] = {"value": 1.0 / one[0], "cores": 1, "seconds_per_product": one[0], "sweeps": one[1]}
        if out["one_thread"]["value"] > best["value"]:
            best = out["one_thread"]
    out.update(value=best["value"], cores=best["cores"],
               sample=f"one whole product of the workload (initial CI and all {best['sweeps']} sweeps actually run) "
                      f"with {best['cores']} BLAS thread(s): {best['seconds_per_product']:.1f} s wall clock; the "
                      f"other thread count is reported beside it")
    return out


def run_reference(args):
    """The reference arm: the CPU oracle, sweep by sweep. A step is one sweep iteration of the
    workload's product (the first step of a product also carries its initial CI); K timed steps run
    products back to back, each for up to max_sweeps iterations, so K = max_sweeps is one whole
    product. value = products completed per second = (steps / sweeps per product) / seconds."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.oracle_threads > 0:  # before numpy loads: its BLAS fixes the thread count then
        for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = str(args.oracle_threads)
    p = workload(args.chi)
    if args.warmup:
        oracle_product(p, args.max_sweeps, max_iters=min(args.warmup, args.max_sweeps))
    done, total, products, per = 0, 0.0, 0, None
    while done < args.steps:
        n = min(args.max_sweeps, args.steps - done)
        t, marks, iters = oracle_product(p, args.max_sweeps, max_iters=n)
        if per is None:
            per = iters if n == args.max_sweeps else args.max_sweeps
        total += t
        done += iters
        products += 1
        if iters < n:  # the product converged early: its remaining steps do not exist
            break
    value = (done / per) / total
    cores = blas_threads()
    sample = (f"each step = one sweep iteration of the oracle's product (the first of each product also runs "
              f"its initial CI); {done} steps timed as {products} product run(s), {per} sweeps per product")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / max(done, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, p),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        log_dir = os.environ.get("ACI_BENCH_LOG_DIR", tempfile.gettempdir())
        self.path = os.path.join(log_dir, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------ our arm

def source_hash(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def recorded_traffic(kernel_class):
    """DRAM bytes per byte of the launch's input block, from a committed ncu summary
    (profiles/traffic.txt: class, source hash, ratio), if the kernel source still matches."""
    f = os.path.join(ROOT, "profiles", "traffic.txt")
    src = {"pivot": "aci_prrlu.cu", "pi": "aci_gemm.cu", "frame": "aci_gemm.cu"}.get(kernel_class)
    if not src or not os.path.exists(f):
        return None
    h = source_hash(os.path.join(ROOT, "paper_2604_00037_gb300", "csrc", src))
    for line in open(f):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel_class and parts[1] == h:
            return float(parts[2])
    return None


def update_order(L, iterations):
    """Local updates of a product in execution order, as pivot-history keys (u, bond)."""
    order = [(0, s - 1) for s in range(L - 1, 0, -1)]
    for it in range(1, iterations + 1):
        order += [(1 + 2 * (it - 1), b) for b in range(L - 1)]
        order += [(2 + 2 * (it - 1), b) for b in range(L - 2, -1, -1)]
    return order


def pivot_work(info, d, max_rank, in_ranks, elem_bytes=8):
    """From one product's pivot history: pivot-search launches, accepted pivots, pivot steps (each
    launch also takes one step that ends in the stop decision unless its block is used up) and the
    algorithmic bytes of the blocks the launches factorise (each read once)."""
    import numpy as np
    hist = info["history"]
    L = len(d)
    cap = [1] + [min(max_rank, 2 ** min(s, 62), int(np.prod(d[:s], dtype=float)), int(np.prod(d[s:], dtype=float)))
                 for s in range(1, L)] + [1]
    ranks = [1] * (L + 1)
    launches = pivots = steps = 0
    nbytes = 0.0
    for (u, b) in update_order(L, info["iterations"]):
        k = len(hist[(u, b)][0])
        if u == 0:  # initial CI of site s = b + 1: (initial-guess rank) x (d_s rank_{s+1})
            s_ = b + 1
            m, n = min(cap[s_], *[r[s_] for r in in_ranks]), d[s_] * ranks[s_ + 1]
        else:
            m, n = ranks[b] * d[b], d[b + 1] * ranks[b + 2]
        ranks[b + 1] = k
        launches += 1
        pivots += k
        steps += k + (0 if k == min(m, n) else 1)
        nbytes += float(m) * n * elem_bytes
    return dict(launches=launches, pivots=pivots, steps=steps, block_bytes=nbytes)


def sample_points(rng, L, d, n):
    import numpy as np
    return rng.integers(0, d, size=(n, L))


def rel_err(y, ref):
    import numpy as np
    return float(np.abs(y - ref).max() / np.abs(ref).max())


def run_time_to_tol(ctx, A, B, a, b, p, args, stream):
    """Device time and sampled error after each sweep: the call with max_sweeps = t, t = 1, 2, ..."""
    import numpy as np
    import torch
    from synthetic.tt import tt_eval
    pts = sample_points(np.random.default_rng(11), len(a), 2, 4000)
    exact = tt_eval(a, pts) * tt_eval(b, pts)
    rows = []
    for t in range(1, args.max_sweeps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        y, info = ctx.elementwise(A, B, "mul", p["tol"], p["max_rank"], max_sweeps=t, overlap=args.overlap,
                                  precision=args.precision, pivot_mode=args.pivot_mode)
        e1.record(stream)
        e1.synchronize()
        err = rel_err(tt_eval([c.cpu().numpy() for c in y], pts), exact)
        rows.append({"sweeps": info["iterations"], "ms": e0.elapsed_time(e1), "rel_err_vs_exact": err,
                     "max_eps_rel": info["max_eps"] / info["scale"], "max_rank": max(info["ranks"])})
        if info["iterations"] < t:
            break
    first = next((r for r in rows if r["rel_err_vs_exact"] <= 1e-8), None)
    return {"target_rel_err": 1e-8, "points": len(pts), "per_sweep": rows,
            "first_sweep_at_target": first["sweeps"] if first else None,
            "ms_at_target": first["ms"] if first else None,
            "note": "a row per max_sweeps = t call (device time of the whole call, CUDA events); the error is "
                    "the max relative error against the exact product on seeded grid points"}


def run_vs_chi(ctx, args, stream):
    """Time per product of the same workload at other input ranks (the metric's time vs chi):
    config 2 with chi from --vs-chi, max_rank 2 chi, tol 1e-10; median of 3 calls after one."""
    import numpy as np
    import torch
    from synthetic.tt import tt_eval
    rows = []
    for chi in [int(c) for c in args.vs_chi.split(",") if c]:
        p = workload(chi)
        a, b = p["inputs"]
        A, B = [torch.from_numpy(c).cuda() for c in a], [torch.from_numpy(c).cuda() for c in b]
        call = lambda: ctx.elementwise(A, B, "mul", p["tol"], p["max_rank"], max_sweeps=args.max_sweeps,
                                       overlap=args.overlap, autotune=bool(args.autotune))
        call()
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            y, info = call()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        pts = sample_points(np.random.default_rng(13), len(a), 2, 4000)
        exact = tt_eval(a, pts) * tt_eval(b, pts)
        rows.append({"chi": chi, "ms_per_product": statistics.median(ts), "iterations": info["iterations"],
                     "max_rank": max(info["ranks"]), "max_eps_rel": info["max_eps"] / info["scale"],
                     "rel_err_vs_exact": rel_err(tt_eval([c.cpu().numpy() for c in y], pts), exact)})
    return rows


def run_cfg3(ctx, args, stream, fp64_peak):
    """The fused d = 8 workload: |psi|^2 psi of a 3D complex field, 12 sites, chi = 128, tol 1e-8,
    max_rank chi, in FP64 and with BF16 digit-plane contractions (plain schedule at d = 8)."""
    import numpy as np
    import torch
    from synthetic import config_inputs
    from synthetic.tt import tt_eval
    p = config_inputs(3, args.cfg3_chi)
    a = p["inputs"][0]
    A = [torch.from_numpy(c).cuda() for c in a]
    pts = sample_points(np.random.default_rng(12), len(a), 8, 4000)
    psi = tt_eval(a, pts)
    exact = (psi.real ** 2 + psi.imag ** 2) * psi
    out = {"workload": f"3D quantics, 12 sites of d = 8 (2^36 points), complex128 500-mode field, chi = "
                       f"{args.cfg3_chi}, |psi|^2 psi, tol {p['tol']:g} rel, max_rank {p['max_rank']}"}
    vals = {}
    prec_list = ["fp64"] + ([f"bf16x{args.mixed_digits}"] if args.mixed_digits else [])
    for prec in prec_list:
        call = lambda prof: ctx.elementwise(A, None, "abs2_mul", p["tol"], p["max_rank"], max_sweeps=args.max_sweeps,
                                            precision=prec, profile=prof)
        call(False)
        ts = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            y, info = call(False)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        _, pinfo = call(True)
        yv = tt_eval([c.cpu().numpy() for c in y], pts)
        vals[prec] = yv
        k = pinfo["kernels"]
        ent = {"ms_per_product": statistics.median(ts), "iterations": info["iterations"],
               "max_rank": max(info["ranks"]), "rel_err_vs_exact": rel_err(yv, exact),
               "classes_ms": {c: k[c]["ms"] for c in k}}
        if prec == "fp64":
            cms = k["frame"]["ms"] + k["pi"]["ms"]
            cfl = k["frame"]["flops"] + k["pi"]["flops"]
            ach = cfl / (cms / 1e3) / 1e12
            ent["roofline_fp64"] = {"bound": "alu", "kernel": "gemm_kernel (frames and Pi)", "achieved": ach,
                                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                                    "peak_source": "FP64 FMA probe (aci_k_fp64_peak), measured in this run"}
        else:
            tms = k["frame"]["ms"] + k["pi"]["ms"]
            tfl = k["frame"]["tensor_flops"] + k["pi"]["tensor_flops"]
            peak, src = measured_peak("bf16_tflops", 1900.0)
            ach = tfl / (tms / 1e3) / 1e12
            ent["rel_err_vs_fp64"] = rel_err(yv, vals["fp64"])
            ent["roofline_tensor"] = {"bound": "tensor", "kernel": "tc_split_kernel + tc_gemm_kernel (frames and Pi)",
                                      "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                                      "peak_source": f"bf16 dense, {src} (burst)",
                                      "note": "BF16 MMA flops issued / device time of the contraction launches"}
        out[prec] = ent
    if len(prec_list) > 1:
        out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_product"] / out[prec_list[1]]["ms_per_product"]
    return out


def _batch_pair(spec):
    from synthetic.fields import batch_config4_pair
    return batch_config4_pair(spec)


def make_batch(n):
    """The batched workload's inputs, generated in a spawned pool (before any GPU call)."""
    import multiprocessing as mp
    from synthetic.fields import batch_config4_spec
    spec = batch_config4_spec(n=n)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"  # one BLAS thread per generator process (inherited by the pool)
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        pairs = pool.map(_batch_pair, spec)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.pop(v, None)
    return spec, pairs, time.time() - t0


def batch_items(spec, pairs):
    import torch
    items = []
    for sp, (a, b) in zip(spec, pairs):
        dt = torch.float32 if sp["dtype"] == "f32" else torch.float64
        items.append(dict(a=[torch.from_numpy(c).to(dt).cuda() for c in a],
                          b=[torch.from_numpy(c).to(dt).cuda() for c in b],
                          op=sp["op"], tol=sp["tol"], max_rank=sp["max_rank"]))
    return items


def run_batch_line(ctx, spec, pairs, gen_s, args, stream, reps=1, streams_list=(1, 0)):
    import numpy as np
    import torch
    items = batch_items(spec, pairs)
    ctx.elementwise_batch(items[: min(4, len(items))], streams=1, max_sweeps=args.max_sweeps)
    out = {}
    for streams, tuned in [(s_, False) for s_ in streams_list] + [(0, True)]:
        label = "one_at_a_time" if streams == 1 else ("concurrent_tuned" if tuned else "concurrent")
        if streams == 0:  # the autotuners' trial calls come first, untimed
            for _ in range(3):
                ctx.elementwise_batch(items, streams=0, max_sweeps=args.max_sweeps, autotune=tuned)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = ctx.elementwise_batch(items, streams=streams, max_sweeps=args.max_sweeps, autotune=tuned)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        out[label] = {"streams": streams if streams else "autotuned", "ms_per_batch": ms,
                      "products_per_s": len(items) / (ms / 1e3),
                      "contraction_tuner": tuned, "statuses": sorted({r[1]["status"] for r in res})}
    return {"workload": f"{len(items)} pairs of 2D interleaved 200-mode Fourier fields, L in [20, 40], chi in "
                        f"[16, 256], even pairs FP64 and odd pairs FP32, a*b / a*conj(b), tol 1e-8 rel, max_rank chi",
            "value": max(out["concurrent"]["products_per_s"], out["concurrent_tuned"]["products_per_s"]),
            "unit": "products/s",
            **out, "speedup": out["one_at_a_time"]["ms_per_batch"] / min(out["concurrent"]["ms_per_batch"],
                                                                          out["concurrent_tuned"]["ms_per_batch"]),
            "input_generation_s": gen_s}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel:
        return run_kernel(args)
    if args.batch:
        return run_batch(args)
    if args.proposer:
        return run_proposer(args)
    if args.scaling:
        return run_scaling(args)
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    batch = seq = None
    if args.batch_line and rank == 0 and world == 1:
        batch = make_batch(args.batch_line)  # spawned pool: before any GPU call
    if args.proposer_line and rank == 0 and world == 1:
        seq = make_sequence(args.proposer_line, 128)  # spawned pool: before any GPU call
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2604_00037_gb300.binding import Context

    p = workload(args.chi)
    a, b = p["inputs"]
    A = [torch.from_numpy(c).cuda() for c in a]
    B = [torch.from_numpy(c).cuda() for c in b]
    ctx = Context(local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    fp64_peak = ctx.fp64_peak()

    def step(profile=False, history=False):
        return ctx.elementwise(A, B, "mul", p["tol"], p["max_rank"], max_sweeps=args.max_sweeps, profile=profile,
                               precision=args.precision, pivot_mode=args.pivot_mode, overlap=args.overlap,
                               history=history, autotune=bool(args.autotune))

    for w in range(args.warmup):
        flush.fill_(w & 0xFF)
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times, infos = [], []
    for k in range(args.steps):
        flush.fill_((k + 7) & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        y, info = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        infos.append(info)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(times)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)

    # One more product with per-launch CUDA events (the library times every kernel on its stream)
    # and the pivot history: the class breakdown and the pivot search's roofline and latency.
    flush.fill_(3)
    _, dinfo = step(profile=True, history=True)
    classes = ("frame", "pi", "pivot", "other")
    kms = {c: dinfo["kernels"][c]["ms"] for c in classes}
    kcnt = {c: dinfo["kernels"][c]["count"] for c in classes}
    kfl = {c: dinfo["kernels"][c]["flops"] for c in classes}
    work = pivot_work(dinfo, [2] * len(a), p["max_rank"], [[1] + [c.shape[2] for c in x] for x in (a, b)])
    dom = max(("frame", "pi", "pivot"), key=lambda c: kms[c])
    achieved = kfl[dom] / (kms[dom] / 1e3) / 1e12
    ratio = recorded_traffic(dom)
    traffic = ratio * work["block_bytes"] / work["launches"] if ratio is not None and dom == "pivot" else None
    wall = dinfo["device_ms"]
    roofline = {"bound": "alu", "kernel": {"frame": "gemm_kernel (frame half-products)",
                                           "pi": "gemm_kernel (Pi block + f)",
                                           "pivot": "pivot search: prrlu_creg_kernel (1D) / prrlu_c2d_kernel (2D) / "
                                                    "prrlu_cta_kernel (single CTA), chosen per launch"}[dom],
                "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                "traffic": traffic,
                "traffic_note": ("DRAM bytes per launch: the ncu ratio of DRAM bytes to input-block bytes "
                                 "(profiles/traffic.txt) times the mean block of this product's launches"
                                 if traffic is not None else "no ncu capture of the current kernel source"),
                "peak_source": f"FP64 FMA probe (aci_k_fp64_peak) measured in this run (nominal "
                               f"{FP64_NOMINAL_TFLOPS} TFLOP/s; no FP64 tensor path on GB300)",
                "share": kms[dom] / wall,
                "profiled_product_ms": wall,
                "classes_ms_per_step": kms, "classes_flops_per_step": kfl, "classes_launches_per_step": kcnt}
    if dom == "pivot":
        roofline["latency"] = {
            "launches": work["launches"], "pivots": work["pivots"], "pivot_steps": work["steps"],
            "us_per_pivot_step": kms["pivot"] * 1e3 / work["steps"],
            "block_bytes": work["block_bytes"],
            "l2_gbs": work["block_bytes"] / (kms["pivot"] / 1e3) / 1e9,
            "note": "each pivot step is one argmax exchange of the sequential search; the blocks (<= 2 MB each) "
                    "are read once per launch, from L2 or HBM: l2_gbs = block bytes / pivot-class time"}

    # end to end: host (pinned) buffers through the C ABI, copies inside the timed region
    ah = [torch.from_numpy(c).pin_memory().numpy() for c in a]
    bh = [torch.from_numpy(c).pin_memory().numpy() for c in b]
    h2d = sum(c.nbytes for c in ah) + sum(c.nbytes for c in bh)
    ekw = dict(max_sweeps=args.max_sweeps, out_memory="host", precision=args.precision, pivot_mode=args.pivot_mode,
               overlap=args.overlap, autotune=bool(args.autotune))
    ctx.elementwise(ah, bh, "mul", p["tol"], p["max_rank"], **ekw)
    e2e_t, d2h = [], 0
    for k in range(max(1, min(args.steps, 3))):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        yh, _ = ctx.elementwise(ah, bh, "mul", p["tol"], p["max_rank"], **ekw)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
        d2h = sum(c.nbytes for c in yh)
    e2e_value = len(e2e_t) / sum(e2e_t)
    if world > 1:
        t = torch.tensor([sum(e2e_t)], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_value = world * len(e2e_t) / float(t.item())

    ttt = run_time_to_tol(ctx, A, B, a, b, p, args, stream) if args.time_to_tol and rank == 0 else None
    vs_chi = run_vs_chi(ctx, args, stream) if args.vs_chi and rank == 0 else None

    # the same workload with the contractions on the tensor cores; errors on 20000 sampled points
    mixed = None
    if args.mixed_digits:
        from synthetic.tt import tt_eval
        prec = f"bf16x{args.mixed_digits}"
        pts = sample_points(np.random.default_rng(8), len(a), 2, 20000)
        exact = tt_eval(a, pts) * tt_eval(b, pts)
        y64 = tt_eval([c.cpu().numpy() for c in y], pts)

        def mstep(profile):
            return ctx.elementwise(A, B, "mul", p["tol"], p["max_rank"], max_sweeps=args.max_sweeps, profile=profile,
                                   precision=prec, overlap=args.overlap)
        mstep(False)
        mt = []
        for k in range(args.steps):
            flush.fill_((k + 3) & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ym, _ = mstep(False)
            e1.record(stream)
            e1.synchronize()
            mt.append(e0.elapsed_time(e1))
        _, minfo = mstep(True)
        yv = tt_eval([c.cpu().numpy() for c in ym], pts)
        k_ = minfo["kernels"]
        tms = k_["frame"]["ms"] + k_["pi"]["ms"]
        tfl = k_["frame"]["tensor_flops"] + k_["pi"]["tensor_flops"]
        peak, src = measured_peak("bf16_tflops", 1900.0)
        ach = tfl / (tms / 1e3) / 1e12
        mixed = {"precision": prec, "value": world * args.steps / (sum(mt) / 1e3), "unit": UNIT,
                 "ms_per_step": sum(mt) / args.steps,
                 "rel_err_vs_exact": rel_err(yv, exact), "rel_err_vs_fp64": float(np.abs(yv - y64).max() / np.abs(exact).max()),
                 "fp64_rel_err_vs_exact": rel_err(y64, exact),
                 "classes_ms_per_step": {c: k_[c]["ms"] for c in classes},
                 "roofline_tensor": {"bound": "tensor", "kernel": "tc_split_kernel + tc_gemm_kernel (frames and Pi)",
                                     "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                                     "peak_source": f"bf16 dense, {src} (burst)",
                                     "note": "BF16 MMA flops issued / device time of the contraction launches"}}

    cfg3 = run_cfg3(ctx, args, stream, fp64_peak) if args.cfg3 and rank == 0 else None
    batch_line = run_batch_line(ctx, *batch, args, stream) if batch is not None else None
    proposer_line = proposer_measure(ctx, seq[0], 128, [1.25], args.max_sweeps, seq[1]) if seq is not None else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_line(p, args)

    last = infos[-1]
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else f"f64 ({args.precision} contractions)",
                "data": "synthetic", "config": config_dict(args, p),
                "result": {"iterations": last["iterations"], "converged": last["converged"],
                           "max_rank": max(last["ranks"]), "max_eps_rel": last["max_eps"] / last["scale"]},
                "roofline": roofline, "fp64_peak_tflops": fp64_peak, "cpu_baseline": cpu,
                "time_to_tol": ttt, "vs_chi": vs_chi, "mixed": mixed, "cfg3": cfg3, "batch": batch_line,
                "proposer": proposer_line,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
