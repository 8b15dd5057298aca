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
# FP64 vector peak of a GB300 (nominal 1.25 TFLOP/s: 152 SMs x ~2 DFMA/clk/SM at ~2.06 GHz);
# a probe on this pool measured 1.197 TFLOP/s of DFMA throughput.
FP64_PEAK_TFLOPS = 1.25
SAMPLE_ITERS = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--chi", type=int, default=128)
    ap.add_argument("--max-sweeps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixed-digits", type=int, default=6, help="BF16 digit planes of the mixed run (0: skip it)")
    ap.add_argument("--precision", default="fp64", help="contractions of the headline run: fp64 or bf16xS")
    ap.add_argument("--pivot-mode", default="full", choices=["full", "rook"])
    ap.add_argument("--overlap", default="auto", choices=["auto", "off", "on"],
                    help="schedule of the sweeps (aci_opts.sweep_overlap)")
    ap.add_argument("--kernel", default="", choices=["", "pi_block", "frame_gemm", "prrlu"],
                    help="time one step-level call of this shape instead of the product (kernel profiling)")
    ap.add_argument("--m", type=int, default=2048)
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--k", type=int, default=256)
    ap.add_argument("--complex", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="time this many independent pairs of the batched workload instead (aci_elementwise_batch)")
    ap.add_argument("--streams", type=int, default=0, help="batch: products in flight (0 = library default)")
    ap.add_argument("--proposer", action="store_true",
                    help="the learned-proposal sequence: train on steps 0-39, compare on 40-59")
    ap.add_argument("--seq-steps", type=int, default=60)
    ap.add_argument("--keep", default="1.25",
                    help="proposer: kept candidates per side = keep x previous rank + 8; a comma list compares several")
    return ap.parse_args()


def _seq_pair(args):
    t, chi = args
    from synthetic.fields import sequence_config5_pair
    return sequence_config5_pair(t, chi)


def run_proposer(args):
    """The learned-proposal sequence (synthetic/fields.py, sequence_config5_pair): products f_t g_t,
    tol 1e-8, max_rank 2 chi. Plain ACI runs steps 0 .. 2/3 of the sequence while recording the
    (features, pivot-or-not) pairs of its left-to-right updates; the network is trained on them with
    the library's kernels (Adam, weighted logistic loss); the remaining steps run with plain ACI and
    with the learned restriction. Reports time per product, the error of both against the exact
    product on 20000 sampled points, and the recall of plain ACI's pivots by the kept candidates."""
    import multiprocessing as mp
    import numpy as np
    nsteps = args.seq_steps
    ntrain = (2 * nsteps) // 3
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:  # before any GPU call
        pairs = pool.map(_seq_pair, [(t, args.chi) for t in range(nsteps)])
    gen_s = time.time() - t0
    print(f"proposer: {nsteps} steps generated in {gen_s:.1f} s", file=sys.stderr, flush=True)
    import torch
    from oracle import mlp
    from paper_2604_00037_gb300.binding import Context
    from synthetic.tt import tt_eval
    ctx = Context(0)
    tol, max_rank = 1e-8, 2 * args.chi
    dev = lambda tt: [torch.from_numpy(c).cuda() for c in tt]
    read = ctx.record_proposer_data(4_000_000)
    for t in range(ntrain):
        a, b = pairs[t]
        ctx.elementwise(dev(a), dev(b), "mul", tol, max_rank, max_sweeps=args.max_sweeps)
    X, y, nrec = read()
    pos = float(y.mean().item())
    P = torch.from_numpy(mlp.init(0, 7)).cuda()
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
    keeps = [float(k) for k in str(args.keep).split(",")]
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
                ycores, info = ctx.elementwise(A, B, "mul", tol, max_rank, max_sweeps=args.max_sweeps,
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
    # recall: of plain ACI's pivots in recorded held-out data, the share the proposer keeps
    read = ctx.record_proposer_data(2_000_000)
    a, b = pairs[nsteps - 1]
    ctx.elementwise(dev(a), dev(b), "mul", tol, max_rank, max_sweeps=args.max_sweeps)
    Xt, yt, _ = read()
    zt = ctx.mlp_forward(Xt, P, fp16=True).cpu().numpy()
    yt = yt.cpu().numpy()
    sub = np.random.default_rng(9)
    zp, zn = zt[yt > 0.5], zt[yt < 0.5]
    zp = zp[sub.permutation(len(zp))[:2000]]
    zn = zn[sub.permutation(len(zn))[:2000]]
    line = {"metric": "learned pivot proposal: ACI time per product at equal error (held-out steps)",
            "unit": "ms/product", "value": summ["proposed"]["ms_per_product"], "higher_is_better": False,
            "dtype": "f64", "data": "synthetic", "n_gpus": 1,
            "config": {"workload": f"{nsteps}-step sequence f_t g_t of 2D interleaved Fourier fields (L=40, d=2, "
                                   f"chi={args.chi}), phases advancing by omega_k t; tol {tol:g}, max_rank {max_rank}; "
                                   f"trained on steps 0-{ntrain - 1}, compared on {ntrain}-{nsteps - 1}",
                       "keep": args.keep, "input_generation_s": gen_s},
            "training": {"records": int(X.shape[0]), "positive_share": pos, "final_loss": loss,
                         "adam_steps": 400, "train_s": train_s},
            **{m: summ[m] for m in modes},
            "speedup": summ["plain"]["ms_per_product"] / summ["proposed"]["ms_per_product"],
            **{f"speedup@{k:g}": summ["plain"]["ms_per_product"] / summ[m]["ms_per_product"]
               for k, m in zip(keeps, modes[1:])},
            "held_out_auc": float((zp[:, None] > zn[None, :]).mean()) if len(zp) and len(zn) else float("nan")}
    print(json.dumps(line), flush=True)
    ctx.close()


def _make_pair(spec):
    from synthetic.fields import batch_config4_pair
    return batch_config4_pair(spec)


def run_batch(args):
    """The batched workload: args.batch pairs of uneven length and rank (synthetic/fields.py,
    batch_config4_spec), FP64, each product exactly as aci_elementwise_ex computes it. Times the
    whole batch through aci_elementwise_batch with one product in flight and with args.streams
    (library default when 0), after a warm-up batch; inputs are device-resident."""
    import multiprocessing as mp
    from synthetic.fields import batch_config4_spec
    spec = batch_config4_spec(n=args.batch)
    t0 = time.time()
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"  # one BLAS thread per generator process (inherited by the pool)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:  # before any GPU call
        pairs = pool.map(_make_pair, spec)
    gen_s = time.time() - t0
    print(f"batch: {len(pairs)} pairs generated in {gen_s:.1f} s", file=sys.stderr, flush=True)
    import torch
    from paper_2604_00037_gb300.binding import Context
    ctx = Context(0)
    items = [dict(a=[torch.from_numpy(c).cuda() for c in a], b=[torch.from_numpy(c).cuda() for c in b],
                  op=sp["op"], tol=sp["tol"], max_rank=sp["max_rank"]) for sp, (a, b) in zip(spec, pairs)]
    out = {}
    for label, streams in (("sequential", 1), ("concurrent", args.streams)):
        ctx.elementwise_batch(items[: min(4, len(items))], streams=streams, max_sweeps=args.max_sweeps)
        torch.cuda.synchronize()
        times = []
        for _ in range(max(1, args.steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            res = ctx.elementwise_batch(items, streams=streams, max_sweeps=args.max_sweeps)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            print(f"batch: {label} streams={streams} {times[-1]:.0f} ms", file=sys.stderr, flush=True)
        ms = statistics.median(times)
        out[label] = {"streams": streams, "ms_per_batch": ms, "products_per_s": len(items) / (ms / 1e3),
                      "statuses": sorted({r[1]["status"] for r in res})}
    line = {"metric": "batched ACI products/s (independent pairs of uneven L and chi)", "unit": "products/s",
            "value": out["concurrent"]["products_per_s"], "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "n_gpus": 1, "steps": args.steps,
            "config": {"workload": f"{len(items)} pairs of 2D interleaved Fourier fields, L in [20, 40], "
                                   f"chi in [16, 256], a*b / a*conj(b), tol 1e-8 rel, max_rank chi",
                       "input_generation_s": gen_s},
            "sequential": out["sequential"], "concurrent": out["concurrent"],
            "speedup": out["sequential"]["ms_per_batch"] / out["concurrent"]["ms_per_batch"]}
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
            "l2": "flushed before every timed step (256 MB write, untimed)",
            "parallelism": f"replicas x{args.gpus}"}


# ------------------------------------------------------------------------------ CPU oracle

def oracle_sample(p, max_sweeps):
    """Time the oracle on the first SAMPLE_ITERS sweeps of the product; extrapolate to a product.

    Returns (estimated seconds per product, sample seconds, threads)."""
    import oracle
    a, b = p["inputs"]
    t0 = time.perf_counter()
    oracle.aci([a, b], "mul", p["tol"], p["max_rank"], maxiter=SAMPLE_ITERS)
    t = time.perf_counter() - t0
    per_product = t * max_sweeps / SAMPLE_ITERS
    return per_product, t


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info()]
        return max(n) if n else 1
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = workload(args.chi)
    for _ in range(args.warmup):
        oracle_sample(p, args.max_sweeps)
    est = []
    for _ in range(args.steps):
        per, t = oracle_sample(p, args.max_sweeps)
        est.append(per)
    value = len(est) / sum(est)
    cores = blas_threads()
    sample = (f"each step: the CPU oracle's initial CI and first {SAMPLE_ITERS} of {args.max_sweeps} sweeps of "
              f"the same product; per-product time = sample time x {args.max_sweeps}/{SAMPLE_ITERS}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
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


def mean_pi_bytes(ranks, d=2):
    """Mean bytes of one Π block (FP64) over the bonds at the final ranks: the input block a
    pivot-search launch reads."""
    nb = len(ranks) - 2
    return sum(8.0 * d * ranks[b] * d * ranks[b + 2] for b in range(nb)) / max(nb, 1)


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
    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
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

    def step(profile):
        return ctx.elementwise(A, B, "mul", p["tol"], p["max_rank"], max_sweeps=args.max_sweeps, profile=profile,
                               precision=args.precision, pivot_mode=args.pivot_mode, overlap=args.overlap)

    for w in range(args.warmup):
        flush.fill_(w & 0xFF)
        step(False)
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
        y, info = step(True)
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

    # per-kernel-class roofline from the library's CUDA events of the timed steps
    classes = ("frame", "pi", "pivot", "other")
    kms = {c: sum(i["kernels"][c]["ms"] for i in infos) for c in classes}
    kcnt = {c: sum(i["kernels"][c]["count"] for i in infos) for c in classes}
    kfl = {c: sum(i["kernels"][c]["flops"] for i in infos) for c in classes}
    dom = max(("frame", "pi", "pivot"), key=lambda c: kms[c])
    achieved = kfl[dom] / (kms[dom] / 1e3) / 1e12
    ratio = recorded_traffic(dom)
    traffic = ratio * mean_pi_bytes(infos[-1]["ranks"]) if ratio is not None and dom == "pivot" else None
    roofline = {"bound": "alu", "kernel": {"frame": "gemm_kernel (frame half-products)",
                                           "pi": "gemm_kernel (Pi block + f)",
                                           "pivot": "prrlu_kernel"}[dom],
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": traffic,
                "traffic_note": ("DRAM bytes per launch: the ncu ratio of DRAM bytes to input-block bytes "
                                 "(profiles/prrlu_creg_kernel_480x480_k240.md) times the mean Π block at the "
                                 "final ranks" if traffic is not None else "no capture of the current kernel source"),
                "peak_source": "FP64 vector peak, nominal 1.25 TFLOP/s (no FP64 tensor path on GB300)",
                "share": kms[dom] / total_ms * (world if world > 1 else 1),
                "classes_ms_per_step": {c: kms[c] / args.steps for c in classes},
                "classes_flops_per_step": {c: kfl[c] / args.steps for c in classes},
                "classes_launches_per_step": {c: kcnt[c] / args.steps for c in classes}}

    # end to end: host (pinned) buffers through the C ABI, copies inside the timed region
    ah = [torch.from_numpy(c).pin_memory().numpy() for c in a]
    bh = [torch.from_numpy(c).pin_memory().numpy() for c in b]
    h2d = sum(c.nbytes for c in ah) + sum(c.nbytes for c in bh)
    ctx.elementwise(ah, bh, "mul", p["tol"], p["max_rank"], max_sweeps=args.max_sweeps, out_memory="host",
                    precision=args.precision, pivot_mode=args.pivot_mode, overlap=args.overlap)
    e2e_t, d2h = [], 0
    for k in range(max(1, min(args.steps, 3))):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        yh, _ = ctx.elementwise(ah, bh, "mul", p["tol"], p["max_rank"], max_sweeps=args.max_sweeps,
                                out_memory="host", precision=args.precision, pivot_mode=args.pivot_mode,
                                overlap=args.overlap)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
        d2h = sum(c.nbytes for c in yh)
    e2e_value = len(e2e_t) / sum(e2e_t)
    if world > 1:
        t = torch.tensor([sum(e2e_t)], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_value = world * len(e2e_t) / float(t.item())

    # the same workload with the contractions on the tensor cores; errors on 20000 sampled points
    mixed = None
    if args.mixed_digits:
        from synthetic.tt import tt_eval
        prec = f"bf16x{args.mixed_digits}"
        rng = np.random.default_rng(8)
        pts = rng.integers(0, 2, size=(20000, len(a)))
        exact = tt_eval(a, pts) * tt_eval(b, pts)
        y64 = tt_eval([c.cpu().numpy() for c in y], pts)

        def mstep(profile):
            return ctx.elementwise(A, B, "mul", p["tol"], p["max_rank"], max_sweeps=args.max_sweeps, profile=profile,
                                   precision=prec, overlap=args.overlap)
        mstep(False)
        mt, minfo = [], []
        for k in range(args.steps):
            flush.fill_((k + 3) & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ym, info = mstep(True)
            e1.record(stream)
            e1.synchronize()
            mt.append(e0.elapsed_time(e1))
            minfo.append(info)
        yv = tt_eval([c.cpu().numpy() for c in ym], pts)
        scale = np.abs(exact).max()
        tms = sum(i["kernels"][c]["ms"] for i in minfo for c in ("frame", "pi"))
        tfl = sum(i["kernels"][c]["tensor_flops"] for i in minfo for c in ("frame", "pi"))
        peak, src = measured_peak("bf16_tflops", 1900.0)
        ach = tfl / (tms / 1e3) / 1e12
        mixed = {"precision": prec, "value": world * args.steps / (sum(mt) / 1e3), "unit": UNIT,
                 "ms_per_step": sum(mt) / args.steps,
                 "rel_err_vs_exact": float(np.abs(yv - exact).max() / scale),
                 "rel_err_vs_fp64": float(np.abs(yv - y64).max() / scale),
                 "fp64_rel_err_vs_exact": float(np.abs(y64 - exact).max() / scale),
                 "classes_ms_per_step": {c: sum(i["kernels"][c]["ms"] for i in minfo) / args.steps for c in classes},
                 "roofline_tensor": {"bound": "tensor", "kernel": "tc_split_kernel + tc_gemm_kernel (frames and Pi)",
                                     "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                                     "peak_source": f"bf16 dense, {src} (burst)",
                                     "note": "BF16 MMA flops issued / device time of the contraction launches"}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per, t = oracle_sample(p, args.max_sweeps)
        cpu = {"value": 1.0 / per, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
               "sample": f"the CPU oracle's initial CI and first {SAMPLE_ITERS} of {args.max_sweeps} sweeps of one "
                         f"product ({t:.1f} s); per-product time = sample x {args.max_sweeps}/{SAMPLE_ITERS}"}

    last = infos[-1]
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else f"f64 ({args.precision} contractions)",
                "data": "synthetic", "config": config_dict(args, p),
                "result": {"iterations": last["iterations"], "converged": last["converged"],
                           "max_rank": max(last["ranks"]), "max_eps_rel": last["max_eps"] / last["scale"]},
                "roofline": roofline, "cpu_baseline": cpu, "mixed": mixed,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
