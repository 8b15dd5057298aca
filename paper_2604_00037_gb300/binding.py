"""ctypes binding of the ACI C ABI (include/aci.h, include/aci_kernels.h).

Argument marshalling only: every step of the method runs in the CUDA library. PyTorch
provides device memory (the library allocates through hooks backed by the caching
allocator) and the stream. The library must have been built (``build.build()``); importing
this module on a machine without it raises, there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import buildlib as _build

# ---------------------------------------------------------------- C structures (mirror aci.h)

ACI_OK, ACI_W_NOT_CONVERGED = 0, 1
ACI_R64, ACI_C128, ACI_R32, ACI_C64 = 0, 1, 2, 3
ACI_MEM_DEVICE, ACI_MEM_HOST = 0, 1
OPS = {"mul": 0, "mul_conj": 1, "abs2_mul": 2, "affine": 3}
TOL_KINDS = {"rel": 0, "abs": 1}
STATUS = {0: "ACI_OK", 1: "ACI_W_NOT_CONVERGED", -1: "ACI_E_ARG", -2: "ACI_E_SHAPE", -3: "ACI_E_DTYPE",
          -4: "ACI_E_ALLOC", -5: "ACI_E_CUDA", -6: "ACI_E_TIMEOUT", -7: "ACI_E_NUMERIC"}


class AciOp(C.Structure):
    _fields_ = [("kind", C.c_int32), ("_pad", C.c_int32), ("c", (C.c_double * 2) * 4)]


class AciTT(C.Structure):
    _fields_ = [("L", C.c_int32), ("dtype", C.c_int32), ("memory", C.c_int32), ("_pad", C.c_int32),
                ("d", C.POINTER(C.c_int32)), ("rank", C.POINTER(C.c_int64)), ("core", C.POINTER(C.c_void_p))]


class AciOpts(C.Structure):
    _fields_ = [("tol_kind", C.c_int32), ("max_sweeps", C.c_int32), ("pivot_mode", C.c_int32),
                ("precision", C.c_int32), ("seed", C.c_uint64), ("init", C.POINTER(AciTT)),
                ("out_memory", C.c_int32), ("profile", C.c_int32), ("batch_streams", C.c_int32),
                ("sweep_overlap", C.c_int32), ("autotune", C.c_int32), ("_pad2", C.c_int32)]


class AciStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("fixed_point", C.c_int32),
                ("L", C.c_int32), ("max_eps", C.c_double), ("scale", C.c_double), ("tau", C.c_double),
                ("device_ms", C.c_double), ("kernel_launches", C.c_int64),
                ("ranks", C.POINTER(C.c_int64)), ("eps", C.POINTER(C.c_double)),
                ("pivot_rows", C.POINTER(C.c_int32)), ("pivot_cols", C.POINTER(C.c_int32)),
                ("kernel_ms", C.c_double * 4), ("kernel_count", C.c_int64 * 4), ("kernel_flops", C.c_double * 4),
                ("tensor_flops", C.c_double * 4), ("hist_rank", C.POINTER(C.c_int32)),
                ("hist_rows", C.POINTER(C.c_int32)), ("hist_cols", C.POINTER(C.c_int32))]

KERNEL_CLASSES = ("frame", "pi", "pivot", "other")

OVERLAP_MODES = {"auto": 0, "off": 1, "on": 2}
PIVOT_MODES = {"full": 0, "rook": 1, "proposed": 2}
PROPOSER_FEATURES = 7

# aci_precision: "fp64", or "bf16xS" for S = 2..8 exact BF16 digit planes on the tensor cores.
PRECISIONS = {"fp64": 0, **{f"bf16x{s}": s for s in range(2, 9)}}


def _precision_code(p) -> int:
    if isinstance(p, str):
        if p not in PRECISIONS:
            raise ValueError(f"unknown precision {p!r}; expected one of {sorted(PRECISIONS)}")
        return PRECISIONS[p]
    return int(p)


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

# Every symbol the headers declare; tests check the library exports each one.
EXPORTS = ["aci_create", "aci_destroy", "aci_last_error", "aci_opts_default", "aci_elementwise",
           "aci_elementwise_ex", "aci_elementwise_batch", "aci_tt_release", "aci_k_frame_gemm", "aci_k_pi_block",
           "aci_k_frame_gemm_prec", "aci_k_pi_block_prec", "aci_k_prrlu", "aci_k_prrlu_rook",
           "aci_k_tt_random", "aci_k_apply_pinv", "aci_k_prrlu_static", "aci_k_reciprocal",
           "aci_k_mlp_param_count", "aci_k_mlp_forward", "aci_k_mlp_grad", "aci_k_mlp_adam",
           "aci_set_proposer", "aci_set_proposer_record", "aci_k_fp64_peak", "aci_set_wait_limits",
           "aci_elementwise_n"]

_lib = None


def lib_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True) -> C.CDLL:
    """Load the in-tree CUDA library (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"ACI CUDA library missing: {_build.LIB}")
        _build.build()
    lib = C.CDLL(_build.LIB)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.aci_create.argtypes = [C.POINTER(vp), C.c_int, vp, ALLOC_FN, FREE_FN, vp]
    lib.aci_destroy.argtypes = [vp]
    lib.aci_destroy.restype = None
    lib.aci_last_error.argtypes = [vp]
    lib.aci_last_error.restype = C.c_char_p
    lib.aci_opts_default.argtypes = [C.POINTER(AciOpts)]
    lib.aci_opts_default.restype = None
    lib.aci_elementwise.argtypes = [vp, C.POINTER(AciTT), C.POINTER(AciTT), AciOp, dbl, i32, C.POINTER(AciTT)]
    lib.aci_elementwise_ex.argtypes = [vp, C.POINTER(AciTT), C.POINTER(AciTT), AciOp, dbl, i32,
                                       C.POINTER(AciOpts), C.POINTER(AciTT), C.POINTER(AciStats)]
    lib.aci_tt_release.argtypes = [vp, C.POINTER(AciTT)]
    lib.aci_elementwise_n.argtypes = [vp, i32, C.POINTER(AciTT), AciOp, dbl, i32, C.POINTER(AciOpts),
                                      C.POINTER(AciTT), C.POINTER(AciStats)]
    lib.aci_elementwise_batch.argtypes = [vp, i32, C.POINTER(AciTT), C.POINTER(AciTT), C.POINTER(AciOp),
                                          C.POINTER(dbl), C.POINTER(i32), C.POINTER(AciOpts), C.POINTER(AciTT),
                                          C.POINTER(AciStats), C.POINTER(i32)]
    lib.aci_k_frame_gemm.argtypes = [vp, i32, vp, vp, i32, i32, i32, vp, vp, i32, i32, vp]
    lib.aci_k_frame_gemm_prec.argtypes = [vp, i32, i32, vp, vp, i32, i32, i32, vp, vp, i32, i32, vp]
    lib.aci_k_pi_block.argtypes = [vp, i32, i32, C.POINTER(vp), C.POINTER(vp), i32, i32,
                                   C.POINTER(i32), AciOp, vp, C.POINTER(dbl)]
    lib.aci_k_pi_block_prec.argtypes = [vp, i32, i32, i32, C.POINTER(vp), C.POINTER(vp), i32, i32,
                                        C.POINTER(i32), AciOp, vp, C.POINTER(dbl)]
    lib.aci_k_prrlu.argtypes = [vp, i32, vp, i32, i32, dbl, i32, vp, vp, vp, vp, vp,
                                C.POINTER(i32), C.POINTER(dbl)]
    lib.aci_k_prrlu_rook.argtypes = lib.aci_k_prrlu.argtypes
    lib.aci_k_tt_random.argtypes = [vp, i32, C.c_uint64, i32, C.POINTER(i32), C.POINTER(i64), C.POINTER(vp)]
    lib.aci_k_apply_pinv.argtypes = [vp, i32, vp, i32, i32, vp, vp, vp, vp]
    lib.aci_k_reciprocal.argtypes = [vp, vp, i32, vp]
    lib.aci_k_prrlu_static.argtypes = [vp, i32, vp, i32, i32, dbl, i32, vp, vp, vp, vp, vp,
                                       C.POINTER(i32), C.POINTER(dbl)]
    lib.aci_k_fp64_peak.argtypes = [vp, i32, i32, C.POINTER(dbl)]
    lib.aci_set_wait_limits.argtypes = [vp, i64, i64]
    lib.aci_k_mlp_param_count.argtypes = [i32]
    lib.aci_set_proposer.argtypes = [vp, vp, i32, C.c_float]
    lib.aci_set_proposer_record.argtypes = [vp, vp, i64, vp]
    lib.aci_k_mlp_forward.argtypes = [vp, i32, i32, vp, vp, i32, vp]
    lib.aci_k_mlp_grad.argtypes = [vp, i32, i32, vp, vp, C.c_float, vp, vp, C.POINTER(dbl)]
    lib.aci_k_mlp_adam.argtypes = [vp, i32, vp, vp, vp, vp, i32, C.c_float, C.c_float, C.c_float, C.c_float]
    for name in EXPORTS:
        if name not in ("aci_destroy", "aci_last_error", "aci_opts_default", "aci_k_mlp_param_count"):
            getattr(lib, name).restype = C.c_int
    lib.aci_k_mlp_param_count.restype = C.c_int64
    _lib = lib
    return lib


class AciError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def make_op(op: str, coef=None) -> AciOp:
    o = AciOp()
    o.kind = OPS[op]
    if coef is not None:
        for i, c in enumerate(coef):
            o.c[i][0] = float(np.real(c))
            o.c[i][1] = float(np.imag(c))
    return o


def _dtype_code(x) -> int:
    import torch
    if isinstance(x, torch.Tensor):
        codes = {torch.float64: ACI_R64, torch.complex128: ACI_C128, torch.float32: ACI_R32,
                 torch.complex64: ACI_C64}
    else:
        codes = {np.dtype(np.float64): ACI_R64, np.dtype(np.complex128): ACI_C128,
                 np.dtype(np.float32): ACI_R32, np.dtype(np.complex64): ACI_C64}
    if x.dtype in codes:
        return codes[x.dtype]
    raise TypeError(f"unsupported dtype {x.dtype}: use float64, complex128, float32 or complex64")


class _TTArg:
    """Keeps the ctypes arrays of one aci_tt alive for the duration of a call."""

    def __init__(self, cores):
        import torch
        self.cores = list(cores)
        L = len(self.cores)
        self.d = (C.c_int32 * L)(*[int(c.shape[1]) for c in self.cores])
        ranks = [int(self.cores[0].shape[0])] + [int(c.shape[2]) for c in self.cores]
        self.rank = (C.c_int64 * (L + 1))(*ranks)
        self.ptrs = (C.c_void_p * L)()
        on_dev = isinstance(self.cores[0], torch.Tensor) and self.cores[0].is_cuda
        for s, c in enumerate(self.cores):
            if isinstance(c, torch.Tensor):
                if not c.is_contiguous():
                    raise ValueError("cores must be contiguous")
                self.ptrs[s] = c.data_ptr()
            else:
                if not c.flags["C_CONTIGUOUS"]:
                    raise ValueError("cores must be C-contiguous")
                self.ptrs[s] = c.ctypes.data
        self.tt = AciTT()
        self.tt.L = L
        self.tt.dtype = _dtype_code(self.cores[0])
        self.tt.memory = ACI_MEM_DEVICE if on_dev else ACI_MEM_HOST
        self.tt.d = C.cast(self.d, C.POINTER(C.c_int32))
        self.tt.rank = C.cast(self.rank, C.POINTER(C.c_int64))
        self.tt.core = C.cast(self.ptrs, C.POINTER(C.c_void_p))


class Context:
    """An ACI context on one CUDA device, ordered on torch's current stream of that device."""

    def __init__(self, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the ACI library needs a CUDA device")
        self.lib = load_library()
        self.device = torch.device("cuda", device)
        self._live = {}

        def _alloc(nbytes, user):
            t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=self.device)
            self._live[t.data_ptr()] = t
            return t.data_ptr()

        def _free(ptr, user):
            self._live.pop(ptr, None)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        self.stream = torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        st = self.lib.aci_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream),
                                 self._alloc_cb, self._free_cb, None)
        if st != ACI_OK:
            raise AciError(st, "aci_create failed")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.aci_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st < 0:
            raise AciError(st, self.lib.aci_last_error(self.handle).decode())
        return st

    # ------------------------------------------------------------ the method
    def elementwise(self, a, b=None, op="mul", tol=1e-10, max_rank=64, *, tol_kind="rel",
                    max_sweeps=20, seed=0, init=None, coef=None, out_memory="device",
                    pivots=False, profile=False, precision="fp64", pivot_mode="full", overlap="auto",
                    history=False, autotune=False):
        """y ~ f(a, b) by ACI. ``a``/``b``: lists of cores (torch CUDA tensors, or numpy arrays
        for host memory; float64 / complex128, or float32 / complex64 widened by the library).
        ``a`` may instead be a list of 1-4 input TTs (``b`` None): aci_elementwise_n, where 3 or 4
        inputs take op "mul" (the product of all).
        ``precision``: "fp64" or "bf16xS" (S = 2..8 digit planes) for the frame and Pi
        contractions. ``overlap``: "auto", "off" or "on" (aci_overlap, the schedule of the
        sweeps). ``history``: record every local update's pivots (aci_stats.hist_*) into
        info["history"], a dict {(u, b): (rows, cols)} with u = 0 for the initial CI and
        u = 1 + 2 (i - 1) + h for half-sweep h of iteration i. Returns (cores, stats dict)."""
        import torch
        extra = None
        if isinstance(a, (list, tuple)) and a and isinstance(a[0], (list, tuple)):
            extra = [_TTArg(x) for x in a]  # several inputs (aci_elementwise_n)
            A, Bt = extra[0], None
        else:
            A = _TTArg(a)
            Bt = _TTArg(b) if b is not None else None
        opts = AciOpts()
        self.lib.aci_opts_default(C.byref(opts))
        opts.tol_kind = TOL_KINDS[tol_kind]
        opts.max_sweeps = int(max_sweeps)
        opts.seed = int(seed)
        opts.out_memory = ACI_MEM_HOST if out_memory == "host" else ACI_MEM_DEVICE
        opts.profile = 1 if profile else 0
        opts.precision = _precision_code(precision)
        opts.pivot_mode = PIVOT_MODES[pivot_mode]
        opts.sweep_overlap = OVERLAP_MODES[overlap]
        opts.autotune = 1 if autotune else 0
        It = None
        if init is not None:
            It = _TTArg(init)
            opts.init = C.pointer(It.tt)
        L = len(A.cores)
        ranks = (C.c_int64 * (L + 1))()
        eps = (C.c_double * max(L - 1, 1))()
        stats = AciStats()
        stats.ranks = C.cast(ranks, C.POINTER(C.c_int64))
        stats.eps = C.cast(eps, C.POINTER(C.c_double))
        prow = pcol = None
        if pivots:
            prow = (C.c_int32 * (max(L - 1, 1) * max_rank))()
            pcol = (C.c_int32 * (max(L - 1, 1) * max_rank))()
            stats.pivot_rows = C.cast(prow, C.POINTER(C.c_int32))
            stats.pivot_cols = C.cast(pcol, C.POINTER(C.c_int32))
        if history:
            nslots, nb = 1 + 2 * int(max_sweeps), max(L - 1, 1)
            hr = np.full(nslots * nb, -1, dtype=np.int32)
            hrows = np.full(nslots * nb * max_rank, -1, dtype=np.int32)
            hcols = np.full(nslots * nb * max_rank, -1, dtype=np.int32)
            stats.hist_rank = hr.ctypes.data_as(C.POINTER(C.c_int32))
            stats.hist_rows = hrows.ctypes.data_as(C.POINTER(C.c_int32))
            stats.hist_cols = hcols.ctypes.data_as(C.POINTER(C.c_int32))
        out = AciTT()
        if extra is not None:
            arr = (AciTT * len(extra))(*[x.tt for x in extra])
            st = self.lib.aci_elementwise_n(self.handle, len(extra), arr, make_op(op, coef), float(tol),
                                            int(max_rank), C.byref(opts), C.byref(out), C.byref(stats))
        else:
            st = self.lib.aci_elementwise_ex(self.handle, C.byref(A.tt), C.byref(Bt.tt) if Bt else None,
                                             make_op(op, coef), float(tol), int(max_rank), C.byref(opts),
                                             C.byref(out), C.byref(stats))
        self._check(st)
        cores = self._take_output(out)
        info = self._info(st, stats, ranks, eps, L)
        if pivots:
            info["pivot_rows"] = [[int(prow[b * max_rank + q]) for q in range(info["ranks"][b + 1])]
                                  for b in range(L - 1)]
            info["pivot_cols"] = [[int(pcol[b * max_rank + q]) for q in range(info["ranks"][b + 1])]
                                  for b in range(L - 1)]
        if history:
            hrows = hrows.reshape(nslots, nb, max_rank)
            hcols = hcols.reshape(nslots, nb, max_rank)
            hr = hr.reshape(nslots, nb)
            info["history"] = {(u, b): (hrows[u, b, :hr[u, b]].copy(), hcols[u, b, :hr[u, b]].copy())
                               for u in range(nslots) for b in range(L - 1) if hr[u, b] >= 0}
        return cores, info

    def _take_output(self, out):
        """Copy an output TT into numpy (host) or torch (device) cores and release it."""
        import torch
        cores = []
        is_c = out.dtype == ACI_C128
        for s in range(out.L):
            shape = (int(out.rank[s]), int(out.d[s]), int(out.rank[s + 1]))
            ptr = out.core[s]
            if out.memory == ACI_MEM_HOST:
                n = int(np.prod(shape))
                ct = C.c_double * (n * (2 if is_c else 1))
                buf = np.frombuffer(ct.from_address(ptr), dtype=np.float64).copy()
                arr = buf.view(np.complex128) if is_c else buf
                cores.append(arr.reshape(shape))
            else:
                raw = self._live[ptr]
                t = raw[: int(np.prod(shape)) * (16 if is_c else 8)]
                t = t.view(torch.complex128 if is_c else torch.float64).view(shape)
                cores.append(t)
        self.lib.aci_tt_release(self.handle, C.byref(out))
        return cores

    @staticmethod
    def _info(st, stats, ranks, eps, L):
        return dict(status=STATUS[st], iterations=stats.iterations, converged=bool(stats.converged),
                    fixed_point=bool(stats.fixed_point), max_eps=stats.max_eps, scale=stats.scale,
                    tau=stats.tau, device_ms=stats.device_ms, kernel_launches=stats.kernel_launches,
                    ranks=[int(ranks[i]) for i in range(L + 1)],
                    eps=[float(eps[i]) for i in range(max(L - 1, 0))],
                    kernels={k: dict(ms=stats.kernel_ms[i], count=int(stats.kernel_count[i]),
                                     flops=stats.kernel_flops[i], tensor_flops=stats.tensor_flops[i])
                             for i, k in enumerate(KERNEL_CLASSES)})

    def elementwise_batch(self, items, *, tol_kind="rel", max_sweeps=20, seed=0, out_memory="device",
                          precision="fp64", pivot_mode="full", streams=0, profile=False, overlap="auto",
                          autotune=False):
        """Independent products in one call. ``items``: list of dicts with keys a, b (None for
        abs2_mul), op, tol, max_rank (and optional coef). Returns a list of (cores, info) with
        info["status"] per product; raises only for call-level errors."""
        n = len(items)
        args = [(_TTArg(it["a"]), _TTArg(it["b"]) if it.get("b") is not None else None) for it in items]
        A = (AciTT * max(n, 1))(*[x[0].tt for x in args])
        has_b = any(x[1] is not None for x in args)
        B = (AciTT * max(n, 1))(*[(x[1].tt if x[1] is not None else AciTT()) for x in args]) if has_b else None
        ops = (AciOp * max(n, 1))(*[make_op(it.get("op", "mul"), it.get("coef")) for it in items])
        tols = (C.c_double * max(n, 1))(*[float(it.get("tol", 1e-10)) for it in items])
        mr = (C.c_int32 * max(n, 1))(*[int(it.get("max_rank", 64)) for it in items])
        opts = AciOpts()
        self.lib.aci_opts_default(C.byref(opts))
        opts.tol_kind = TOL_KINDS[tol_kind]
        opts.max_sweeps = int(max_sweeps)
        opts.seed = int(seed)
        opts.out_memory = ACI_MEM_HOST if out_memory == "host" else ACI_MEM_DEVICE
        opts.profile = 1 if profile else 0
        opts.precision = _precision_code(precision)
        opts.pivot_mode = PIVOT_MODES[pivot_mode]
        opts.batch_streams = int(streams)
        opts.sweep_overlap = OVERLAP_MODES[overlap]
        opts.autotune = 1 if autotune else 0
        outs = (AciTT * max(n, 1))()
        stats = (AciStats * max(n, 1))()
        keep = []
        for i, x in enumerate(args):
            L = len(x[0].cores)
            rk = (C.c_int64 * (L + 1))()
            ep = (C.c_double * max(L - 1, 1))()
            stats[i].ranks = C.cast(rk, C.POINTER(C.c_int64))
            stats[i].eps = C.cast(ep, C.POINTER(C.c_double))
            keep.append((rk, ep, L))
        status = (C.c_int32 * max(n, 1))()
        st = self.lib.aci_elementwise_batch(self.handle, n, A, B, ops, tols, mr, C.byref(opts), outs, stats, status)
        results = []
        for i in range(n):
            rk, ep, L = keep[i]
            if status[i] < 0:
                results.append((None, dict(status=STATUS.get(status[i], status[i]))))
                continue
            cores = self._take_output(outs[i])
            results.append((cores, self._info(status[i], stats[i], rk, ep, L)))
        if st < 0 and all(status[i] >= 0 for i in range(n)):
            self._check(st)
        return results

    # ------------------------------------------------------------ step-level entry points
    def frame_gemm(self, A, B, arows=None, bcols=None, M=None, K=None, N=None, precision="fp64"):
        """C = A[arows, :K] @ B[:K, bcols] on device tensors (A, B row-major 2-D)."""
        import torch
        M = int(arows.numel()) if arows is not None else (M or A.shape[0])
        N = int(bcols.numel()) if bcols is not None else (N or B.shape[1])
        K = K or A.shape[1]
        Cm = torch.empty((M, N), dtype=A.dtype, device=A.device)
        self._check(self.lib.aci_k_frame_gemm_prec(
            self.handle, _dtype_code(A), _precision_code(precision), A.data_ptr(), arows.data_ptr() if arows is not None else None,
            M, K, A.shape[1], B.data_ptr(), bcols.data_ptr() if bcols is not None else None, N, B.shape[1],
            Cm.data_ptr()))
        return Cm

    def pi_block(self, As, Bs, op="mul", coef=None, precision="fp64"):
        """Pi = f(A^0 B^0, A^1 B^1) entrywise; returns (Pi, max|Pi|)."""
        import torch
        n = len(As)
        M, N = As[0].shape[0], Bs[0].shape[1]
        Pi = torch.empty((M, N), dtype=As[0].dtype, device=As[0].device)
        Ap = (C.c_void_p * n)(*[a.data_ptr() for a in As])
        Bp = (C.c_void_p * n)(*[b.data_ptr() for b in Bs])
        Ks = (C.c_int32 * n)(*[a.shape[1] for a in As])
        mx = C.c_double()
        self._check(self.lib.aci_k_pi_block_prec(self.handle, _dtype_code(As[0]), _precision_code(precision),
                                                 n, Ap, Bp, M, N, Ks, make_op(op, coef), Pi.data_ptr(),
                                                 C.byref(mx)))
        return Pi, mx.value

    def prrlu(self, M, tau, chimax, with_lu=True, mode="full"):
        """Algorithm 2 on a device matrix (``mode`` "full" or "rook"); returns dict(I, J, D, L, U, k, eps)."""
        import torch
        m, n = M.shape
        kc = min(m, n, chimax)
        pr = torch.empty(kc, dtype=torch.int32, device=M.device)
        pc = torch.empty(kc, dtype=torch.int32, device=M.device)
        D = torch.empty(kc, dtype=M.dtype, device=M.device)
        Lm = torch.zeros((kc, m), dtype=M.dtype, device=M.device) if with_lu else None
        Um = torch.zeros((kc, n), dtype=M.dtype, device=M.device) if with_lu else None
        k = C.c_int32()
        eps = C.c_double()
        fn = self.lib.aci_k_prrlu_rook if mode == "rook" else self.lib.aci_k_prrlu
        self._check(fn(self.handle, _dtype_code(M), M.contiguous().data_ptr(), m, n,
                       float(tau), int(chimax), pr.data_ptr(), pc.data_ptr(), D.data_ptr(),
                       Lm.data_ptr() if with_lu else None, Um.data_ptr() if with_lu else None,
                       C.byref(k), C.byref(eps)))
        kk = k.value
        out = dict(I=pr[:kk].cpu().numpy(), J=pc[:kk].cpu().numpy(), D=D[:kk].cpu().numpy(), k=kk,
                   eps=eps.value)
        if with_lu:
            out["L"] = Lm[:kk].T.cpu().numpy()  # column-major m x kcap stored as kcap rows of length m
            out["U"] = Um[:kk].cpu().numpy()
        return out

    # ------------------------------------------------------------ learned proposer
    def set_proposer(self, params, keep=1.25):
        """Use the network `params` (device float32, kept alive here) for pivot_mode="proposed"."""
        self._proposer = params
        self._check(self.lib.aci_set_proposer(self.handle, params.data_ptr() if params is not None else None,
                                              PROPOSER_FEATURES, float(keep)))

    def record_proposer_data(self, capacity):
        """Start recording (features, label) pairs of full left-to-right updates; returns a reader."""
        import torch
        buf = torch.zeros((capacity, PROPOSER_FEATURES + 1), dtype=torch.float32, device=self.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        self._record = (buf, cnt)
        self._check(self.lib.aci_set_proposer_record(self.handle, buf.data_ptr(), capacity, cnt.data_ptr()))

        def read(stop=True):
            n = min(int(cnt.item()), capacity)
            if stop:
                self._check(self.lib.aci_set_proposer_record(self.handle, None, 0, None))
            return buf[:n, :PROPOSER_FEATURES].clone(), buf[:n, PROPOSER_FEATURES].clone(), int(cnt.item())
        return read

    # ------------------------------------------------------------ pivot-proposer network
    def mlp_param_count(self, F):
        return int(self.lib.aci_k_mlp_param_count(int(F)))

    def mlp_forward(self, X, params, fp16=False):
        """Logits of the n rows of X (torch float32, n x F, device)."""
        import torch
        n, F = X.shape
        z = torch.empty(n, dtype=torch.float32, device=X.device)
        self._check(self.lib.aci_k_mlp_forward(self.handle, n, F, X.contiguous().data_ptr(), params.data_ptr(),
                                               1 if fp16 else 0, z.data_ptr()))
        return z

    def mlp_grad(self, X, y, params, pos_weight=1.0):
        """(loss, gradient) of the mean weighted logistic loss; y float32 0/1 on the device."""
        import torch
        n, F = X.shape
        g = torch.empty_like(params)
        loss = C.c_double()
        self._check(self.lib.aci_k_mlp_grad(self.handle, n, F, X.contiguous().data_ptr(), y.contiguous().data_ptr(),
                                            float(pos_weight), params.data_ptr(), g.data_ptr(), C.byref(loss)))
        return loss.value, g

    def mlp_adam(self, params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        """One Adam step in place on params, m, v (device float32)."""
        self._check(self.lib.aci_k_mlp_adam(self.handle, params.numel(), params.data_ptr(), grad.data_ptr(),
                                            m.data_ptr(), v.data_ptr(), int(t), float(lr), float(beta1),
                                            float(beta2), float(eps)))

    def tt_random(self, seed, ranks, dims, complex_values=False):
        import torch
        dt = torch.complex128 if complex_values else torch.float64
        L = len(dims)
        cores = [torch.empty((ranks[s], dims[s], ranks[s + 1]), dtype=dt, device=self.device) for s in range(L)]
        d = (C.c_int32 * L)(*dims)
        r = (C.c_int64 * (L + 1))(*ranks)
        p = (C.c_void_p * L)(*[c.data_ptr() for c in cores])
        self._check(self.lib.aci_k_tt_random(self.handle, ACI_C128 if complex_values else ACI_R64,
                                             int(seed), L, d, r, p))
        return cores

    def set_wait_limits(self, exchange_polls=0, pipeline_polls=0):
        """Bound the device-side waits of later calls to that many polls (0: the defaults)."""
        self._check(self.lib.aci_set_wait_limits(self.handle, int(exchange_polls), int(pipeline_polls)))

    def fp64_peak(self, blocks=None, iters=4096):
        """Measured FP64 fused multiply-add throughput of this GPU in TFLOP/s (aci_k_fp64_peak);
        by default 8 CTAs of 512 threads per SM."""
        import torch
        if blocks is None:
            blocks = 8 * torch.cuda.get_device_properties(self.device).multi_processor_count
        t = C.c_double()
        self._check(self.lib.aci_k_fp64_peak(self.handle, int(blocks), int(iters), C.byref(t)))
        return t.value

    def reciprocal(self, x):
        """1/x with the reciprocal of the pivot search (x: float64 CUDA tensor)."""
        import torch
        y = torch.empty_like(x)
        self._check(self.lib.aci_k_reciprocal(self.handle, x.data_ptr(), x.numel(), y.data_ptr()))
        return y

    def apply_pinv(self, T, LI, D, UJ):
        import torch
        R, k = T.shape
        Y = torch.empty_like(T)
        self._check(self.lib.aci_k_apply_pinv(self.handle, _dtype_code(T), T.data_ptr(), R, k,
                                              LI.contiguous().data_ptr(), D.contiguous().data_ptr(),
                                              UJ.contiguous().data_ptr(), Y.data_ptr()))
        return Y
