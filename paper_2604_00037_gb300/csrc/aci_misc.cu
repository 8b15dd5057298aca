// Output assembly (CI-canonical form, Eq. (ycicanonical): Y_l = T_l P_l^-1), the random
// initial guess of Algorithm 1, and the end-of-iteration test of Algorithm 1.
#include <algorithm>

#include "aci_internal.h"

namespace aci {

namespace {

// ---------------------------------------------------------------- Y = T P^-1
// P = LI D UJ (LI unit lower, UJ unit upper, in pivot order). For one row x of T:
//   w UJ = x   (forward:  w_q = x_q - sum_{p<q} w_p UJ[p,q])
//   z = w D^-1 (D_p = 0 is read as D_p^-1 = 0)
//   y LI = z   (backward: y_p = z_p - sum_{q>p} y_q LI[q,p])
// Each thread owns one row and keeps it in the output row (global, L1-resident).
template <class T, class FT, class FLI, class FUJ, class FD>
__device__ void solve_row(FT xval, int k, FLI li, FUJ uj, FD dv, T* y) {
    for (int q = 0; q < k; ++q) {
        T acc = xval(q);
        for (int p = 0; p < q; ++p) acc = s_fms(y[p], uj(p, q), acc);
        y[q] = acc;
    }
    for (int p = 0; p < k; ++p) {
        const T dp = dv(p);
        y[p] = s_iszero(dp) ? s_zero(T()) : s_div(y[p], dp);
    }
    for (int p = k - 1; p >= 0; --p) {
        T acc = y[p];
        for (int q = p + 1; q < k; ++q) acc = s_fms(y[q], li(q, p), acc);
        y[p] = acc;
    }
}

template <class T>
__global__ void assemble_kernel(AssembleArgs<T> a) {
    const int s = blockIdx.y;
    const int L = a.L;
    const int* chi = a.chi;
    const int ds = a.d[s];
    const int R = chi[s] * ds;                      // rows of Y_s: (alpha, sigma_s)
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int kout = chi[s + 1];                    // columns of Y_s
    T* y = a.Y[s] + (size_t)r * kout;
    // T_s row r: s = 0 -> Pi_0[sigma, J_1]; s >= 1 -> Pi_{s-1}[I_{s-1}[alpha], (sigma, :)].
    const T* Pi;
    size_t rowoff;
    const int* colmap = nullptr;
    int coloff = 0;
    if (s == 0) {
        const BondBuf<T>& b0 = a.bonds[0];
        const int n0 = a.d[1] * chi[2];
        Pi = b0.Pi;
        rowoff = (size_t)r * n0;
        colmap = b0.pcol;
    } else {
        const BondBuf<T>& bp = a.bonds[s - 1];
        const int nprev = ds * chi[s + 1];
        const int alpha = r / ds, sigma = r % ds;
        Pi = bp.Pi;
        rowoff = (size_t)bp.prow[alpha] * nprev;
        coloff = sigma * kout;
    }
    auto xval = [&](int q) -> T { return Pi[rowoff + (colmap ? colmap[q] : coloff + q)]; };
    if (s == L - 1) {  // Y_{L-1} = T_{L-1}
        for (int q = 0; q < kout; ++q) y[q] = xval(q);
        return;
    }
    const BondBuf<T>& bs = a.bonds[s];
    auto li = [&](int q, int p) -> T { return bs.Lm[(size_t)p * bs.Lld + bs.prow[q]]; };
    auto uj = [&](int p, int q) -> T { return bs.Um[(size_t)p * bs.Uld + bs.pcol[q]]; };
    auto dv = [&](int p) -> T { return bs.D[p]; };
    solve_row<T>(xval, kout, li, uj, dv, y);
}

// The same solves with one warp per output row: lane l holds the row's
// columns l, l + 32, ... in registers, and both solves run column by column, so that the updates of
// a step are independent multiply-adds across lanes instead of one thread's chain of k^2 dependent
// ones. Forward: once w_p is final it goes to every lane by a shuffle and each lane subtracts
// w_p UJ[p, q] from its columns q > p (per column the terms come in ascending p, as in
// solve_row). Backward: y_q, final once every q' > q is applied, goes out the same way and each
// lane subtracts y_q LI[q, p] from its p < q (terms in descending q). Column groups of 32 that are
// already final skip the step as a whole (a warp-wide FP64 instruction holds the pipe whatever its
// active lanes). The CTA's 8 warps (8 rows of one site) share AT rows of UJ (columns of LI) at a
// time, gathered into shared memory.
constexpr int AT = 16;       // rows of UJ / columns of LI per shared-memory tile
constexpr int AWARPS = 8;
constexpr int AROWS = 1;     // output rows per warp

template <class T, int JM>
__device__ __forceinline__ T pick(const T (&v)[JM], int j) {
    T r = v[0];
#pragma unroll
    for (int i = 1; i < JM; ++i)
        if (i == j) r = v[i];
    return r;
}
__device__ __forceinline__ double shfl_val(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ cplx shfl_val(cplx v, int src) {
    return mkc(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}

template <class T, int JM>
__global__ void __launch_bounds__(AWARPS * 32) assemble_warp_kernel(AssembleArgs<T> a, int kpad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);  // [AT][kpad]
    const int s = blockIdx.y;
    const int L = a.L;
    const int* chi = a.chi;
    const int ds = a.d[s];
    const int R = chi[s] * ds;
    const int k = chi[s + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rbase = blockIdx.x * (AWARPS * AROWS);
    if (rbase >= R) return;  // the whole CTA alike
    // rows of this warp (rl < 0: none)
    int rows[AROWS];
#pragma unroll
    for (int w = 0; w < AROWS; ++w) {
        const int r = rbase + warp * AROWS + w;
        rows[w] = r < R ? r : -1;
    }
    // T_s rows: s = 0 -> Pi_0[sigma, J_1]; s >= 1 -> Pi_{s-1}[I_{s-1}[alpha], (sigma, :)]
    T acc[AROWS][JM];
#pragma unroll
    for (int w = 0; w < AROWS; ++w) {
        const int r = rows[w];
#pragma unroll
        for (int j = 0; j < JM; ++j) {
            const int q = lane + 32 * j;
            T x = s_zero(T());
            if (r >= 0 && q < k) {
                if (s == 0) {
                    const BondBuf<T>& b0 = a.bonds[0];
                    x = b0.Pi[(size_t)r * (a.d[1] * chi[2]) + b0.pcol[q]];
                } else {
                    const BondBuf<T>& bp = a.bonds[s - 1];
                    const int alpha = r / ds, sigma = r - alpha * ds;
                    x = bp.Pi[(size_t)bp.prow[alpha] * (ds * k) + sigma * k + q];
                }
            }
            acc[w][j] = x;
        }
    }
    if (s < L - 1) {
        const BondBuf<T>& bs = a.bonds[s];
        // forward: w UJ = x
        for (int p0 = 0; p0 < k; p0 += AT) {
            const int np = min(AT, k - p0);
            __syncthreads();
            for (int e = threadIdx.x; e < np * k; e += AWARPS * 32) {
                const int pp = e / k, q = e - pp * k;
                tile[pp * kpad + q] = bs.Um[(size_t)(p0 + pp) * bs.Uld + bs.pcol[q]];
            }
            __syncthreads();
            for (int pp = 0; pp < np; ++pp) {
                const int p = p0 + pp;
                const int jp = p >> 5, lp = p & 31;
#pragma unroll
                for (int w = 0; w < AROWS; ++w) {
                    const T wp = shfl_val(pick<T, JM>(acc[w], jp), lp);
#pragma unroll
                    for (int j = 0; j < JM; ++j) {
                        if (32 * j + 31 <= p || 32 * j >= k) continue;  // warp-uniform: group done or empty
                        const int q = lane + 32 * j;
                        if (q > p && q < k) acc[w][j] = s_fms(wp, tile[pp * kpad + q], acc[w][j]);
                    }
                }
            }
        }
        // z = w D^-1
#pragma unroll
        for (int j = 0; j < JM; ++j) {
            const int q = lane + 32 * j;
            if (q < k) {
                const T dq = bs.D[q];
#pragma unroll
                for (int w = 0; w < AROWS; ++w) acc[w][j] = s_iszero(dq) ? s_zero(T()) : s_div(acc[w][j], dq);
            }
        }
        // backward: y LI = z, columns q = k-1 .. 0
        for (int qhi = k; qhi > 0; qhi -= AT) {
            const int q0 = max(0, qhi - AT), nq = qhi - q0;
            __syncthreads();
            for (int e = threadIdx.x; e < nq * k; e += AWARPS * 32) {
                const int qq = e / k, p = e - qq * k;
                tile[qq * kpad + p] = bs.Lm[(size_t)p * bs.Lld + bs.prow[q0 + qq]];
            }
            __syncthreads();
            for (int qq = nq - 1; qq >= 0; --qq) {
                const int q = q0 + qq;
                const int jq = q >> 5, lq = q & 31;
#pragma unroll
                for (int w = 0; w < AROWS; ++w) {
                    const T yq = shfl_val(pick<T, JM>(acc[w], jq), lq);
#pragma unroll
                    for (int j = 0; j < JM; ++j) {
                        if (32 * j >= q) continue;  // warp-uniform: group done
                        const int p = lane + 32 * j;
                        if (p < q) acc[w][j] = s_fms(yq, tile[qq * kpad + p], acc[w][j]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int w = 0; w < AROWS; ++w) {
        const int r = rows[w];
        if (r < 0) continue;
        T* y = a.Y[s] + (size_t)r * k;
#pragma unroll
        for (int j = 0; j < JM; ++j) {
            const int q = lane + 32 * j;
            if (q < k) y[q] = acc[w][j];
        }
    }
}

template <class T>
__global__ void apply_pinv_kernel(const T* Tm, int R, int k, const T* LI, const T* D, const T* UJ, T* Y) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    auto xval = [&](int q) -> T { return Tm[(size_t)r * k + q]; };
    auto li = [&](int q, int p) -> T { return LI[(size_t)q * k + p]; };
    auto uj = [&](int p, int q) -> T { return UJ[(size_t)p * k + q]; };
    auto dv = [&](int p) -> T { return D[p]; };
    solve_row<T>(xval, k, li, uj, dv, Y + (size_t)r * k);
}

// ---------------------------------------------------------------- SplitMix64 initial guess
// Output c of the stream with seed s: mix(s + (c + 1) * 0x9E3779B97F4A7C15), mix being the
// SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014). Uniform in [-1, 1): (z >> 11) 2^-52 - 1.
__device__ __forceinline__ double sm64_uniform(unsigned long long seed, unsigned long long c) {
    unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * 0x1p-52 - 1.0;
}
__device__ __forceinline__ void sm64_fill(double* p, unsigned long long seed, unsigned long long e) {
    *p = sm64_uniform(seed, e);
}
__device__ __forceinline__ void sm64_fill(cplx* p, unsigned long long seed, unsigned long long e) {
    *p = mkc(sm64_uniform(seed, 2 * e), sm64_uniform(seed, 2 * e + 1));
}

template <class T>
__global__ void tt_random_kernel(unsigned long long seed, long long off, long long count, T* core) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x)
        sm64_fill(core + e, seed, (unsigned long long)(off + e));
}

// ---------------------------------------------------------------- end-of-iteration test
__global__ void iter_check_kernel(int L, const int* chi, int* chi_prev, int* const* pcol,
                                  int* const* jprev, const double* eps_lr, const double* eps_rl,
                                  const unsigned long long* smax, const int* err, IterFlags* flags,
                                  int snapshot_only) {
    __shared__ int s_grew, s_diff;
    __shared__ double s_emax;
    if (threadIdx.x == 0) { s_grew = 0; s_diff = 0; s_emax = 0.0; }
    __syncthreads();
    if (!snapshot_only) {
        for (int s = 1 + threadIdx.x; s < L; s += blockDim.x)
            if (chi[s] > chi_prev[s]) atomicOr(&s_grew, 1);
        for (int b = threadIdx.x; b < L - 1; b += blockDim.x) {
            const double e = fmax(eps_lr[b], eps_rl[b]);
            // non-negative doubles order like their bit patterns
            atomicMax(reinterpret_cast<unsigned long long*>(&s_emax), (unsigned long long)__double_as_longlong(e));
        }
        // fixed point: every J set (positions, in order) equal to the previous iteration's
        for (int b = 0; b < L - 1; ++b) {
            const int k = chi[b + 1];
            if (k != chi_prev[b + 1]) { if (threadIdx.x == 0) s_diff = 1; continue; }
            for (int q = threadIdx.x; q < k; q += blockDim.x)
                if (pcol[b][q] != jprev[b][q]) s_diff = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && !snapshot_only) {
        flags->grew = s_grew;
        flags->fixed = s_diff ? 0 : 1;
        flags->emax = s_emax;
        flags->S = __longlong_as_double((long long)*smax);
        flags->err = *err;
    }
    __syncthreads();
    // snapshot ranks and J sets for the next iteration's comparison
    for (int s = threadIdx.x; s <= L; s += blockDim.x) chi_prev[s] = chi[s];
    for (int b = 0; b < L - 1; ++b) {
        const int k = chi[b + 1];
        for (int q = threadIdx.x; q < k; q += blockDim.x) jprev[b][q] = pcol[b][q];
    }
}

// ---------------------------------------------------------------- gathers of the overlapped sweep
template <class T>
__global__ void __launch_bounds__(256) gather_kernel(GatherArgs<T> a) {
    // launched early behind the previous pivot search (programmatic dependent launch): wait for it
    // before reading its pivots; then let the next pivot search start launching (it waits for this
    // grid's completion before it reads anything)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const GatherJob<T>& j = a.job[blockIdx.y];
    const int rows = dimv(j.rows, a.chi), cols = dimv(j.cols, a.chi);
    const int sld = dimv(j.sld, a.chi), dld = dimv(j.dld, a.chi);
    const int cblk = j.cblk.mul ? dimv(j.cblk, a.chi) : 0;
    const int cstride = j.cblk.mul ? dimv(j.cstride, a.chi) : 0;
    const int n = rows * cols;  // < 2^31: the host rejects larger blocks
    unsigned long long mk = 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int r = e / cols, c = e - r * cols;  // 32-bit division (a 64-bit one costs several times more)
        const T v = j.src[(size_t)gather_row(j.ridx, j.rblk, r) * sld + gather_col(j.cidx, cblk, cstride, c)];
        j.dst[(size_t)r * dld + c] = v;
        const unsigned long long k = key_of(v);
        mk = k > mk ? k : mk;
    }
    if (a.smax && (int)blockIdx.y == a.smax_job) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long ov = __shfl_xor_sync(0xffffffffu, mk, off);
            mk = ov > mk ? ov : mk;
        }
        if ((threadIdx.x & 31) == 0 && mk) {
            const double mag = key_to_mag(__longlong_as_double((long long)mk), T());
            atomicMax(a.smax, (unsigned long long)__double_as_longlong(mag));
        }
    }
}

// ---------------------------------------------------------------- pivot history (diagnostics)
// One local update's pivots into the history record: slot h.slot when >= 0, else the slot of
// half-sweep h.half of the current iteration, 1 + 2 (*iter - 1) + half, with *iter the device
// iteration counter that hist_tick_kernel advances at the start of every iteration.
__global__ void hist_kernel(HistArgs h) {
    const int slot = h.slot >= 0 ? h.slot : 1 + 2 * (*h.iter - 1) + h.half;
    if (slot < 0 || slot >= h.nslots) return;
    const int k = h.chi[h.kidx];
    const size_t u = (size_t)slot * h.nb + h.b;
    if (threadIdx.x == 0) h.rank[u] = k;
    for (int q = threadIdx.x; q < k && q < h.kstride; q += blockDim.x) {
        h.rows[u * h.kstride + q] = h.prow[q];
        h.cols[u * h.kstride + q] = h.pcol[q];
    }
}
__global__ void hist_tick_kernel(int* iter) { *iter += 1; }

// ---------------------------------------------------------------- FP32 inputs
// FP32 / complex64 input cores widened to FP64 / complex128 (exact: every float is a double).
__global__ void promote_kernel(const float* src, long long n, double* dst) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dst[e] = (double)src[e];
}

// ---------------------------------------------------------------- FP64 throughput probe
// Independent chains of FP64 fused multiply-adds per thread: the FP64 pipe's issue rate, the
// denominator of the FP64 rooflines. The chains are seeded from the inputs and summed into out[]
// so that no multiply-add can be removed.
constexpr int kProbeChains = 8;
__global__ void __launch_bounds__(512) fp64_probe_kernel(const double* seed, int iters, double* out) {
    double x[kProbeChains];
    const double a = seed[0], b = seed[1];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = a + (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], b, a);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == 12345.6789) out[blockIdx.x] = s;  // practically never taken; keeps the chains live
}

}  // namespace

void launch_hist(const HistArgs& h, cudaStream_t st) { hist_kernel<<<1, 256, 0, st>>>(h); }
void launch_hist_tick(int* iter, cudaStream_t st) { hist_tick_kernel<<<1, 1, 0, st>>>(iter); }

void launch_promote(const float* src, long long n, double* dst, cudaStream_t st) {
    if (n <= 0) return;
    const long long nb = std::min<long long>((n + 255) / 256, 4096);
    promote_kernel<<<(int)nb, 256, 0, st>>>(src, n, dst);
}

double fp64_probe_flops(int blocks, int iters) {
    return 2.0 * kProbeChains * 512.0 * (double)blocks * (double)iters;
}
void launch_fp64_probe(const double* seed, int blocks, int iters, double* out, cudaStream_t st) {
    fp64_probe_kernel<<<blocks, 512, 0, st>>>(seed, iters, out);
}

template <class T>
void launch_gather(const GatherArgs<T>& a, long long max_elems, int num_sms, cudaStream_t st) {
    const long long want = (max_elems + 1023) / 1024;
    const int bx = (int)std::max(1LL, std::min(want, (long long)num_sms * 4));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(bx, a.njobs);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = prrlu_pdl_mode();
    cudaLaunchKernelEx(&cfg, gather_kernel<T>, a);  // errors surface at the sweep's next check
}

template <class T>
void launch_assemble(const AssembleArgs<T>& a, int Rmax, int Kmax, cudaStream_t st) {
    // the warp-per-row kernel up to rank 256 (8 columns per lane), one thread per row above
    const int jm = (Kmax + 31) / 32;
    void (*fn)(AssembleArgs<T>, int) = nullptr;
    if (jm <= 1) fn = assemble_warp_kernel<T, 1>;
    else if (jm <= 2) fn = assemble_warp_kernel<T, 2>;
    else if (jm <= 4) fn = assemble_warp_kernel<T, 4>;
    else if (jm <= 8) fn = assemble_warp_kernel<T, 8>;
    if (fn) {
        const int kpad = std::max(1, Kmax);
        const size_t smem = sizeof(T) * (size_t)AT * kpad;  // <= 64 KB (complex, rank 256)
        // once per product; a failure here surfaces as the launch's error
        if (cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return;
        dim3 grid((Rmax + AWARPS * AROWS - 1) / (AWARPS * AROWS), a.L);
        fn<<<grid, AWARPS * 32, smem, st>>>(a, kpad);
        return;
    }
    const int nt = 64;
    dim3 grid((Rmax + nt - 1) / nt, a.L);
    assemble_kernel<T><<<grid, nt, 0, st>>>(a);
}

template <class T>
void launch_apply_pinv(const T* Tm, int R, int k, const T* LI, const T* D, const T* UJ, T* Y,
                       cudaStream_t st) {
    if (R <= 0) return;
    const int nt = 64;
    apply_pinv_kernel<T><<<(R + nt - 1) / nt, nt, 0, st>>>(Tm, R, k, LI, D, UJ, Y);
}

template <class T>
void launch_tt_random(uint64_t seed, int L, const long long* off, const long long* count,
                      T* const* cores, cudaStream_t st) {
    for (int s = 0; s < L; ++s) {
        if (count[s] <= 0) continue;
        const int nt = 256;
        long long nb = (count[s] + nt - 1) / nt;
        if (nb > 4096) nb = 4096;
        tt_random_kernel<T><<<(int)nb, nt, 0, st>>>(seed, off[s], count[s], cores[s]);
    }
}

void launch_iter_check(int L, const int* chi, int* chi_prev, int* const* pcol, int* const* jprev,
                       const double* eps_lr, const double* eps_rl, const unsigned long long* smax,
                       const int* err, IterFlags* flags, int snapshot_only, cudaStream_t st) {
    iter_check_kernel<<<1, 256, 0, st>>>(L, chi, chi_prev, pcol, jprev, eps_lr, eps_rl, smax, err,
                                         flags, snapshot_only);
}

template void launch_gather<double>(const GatherArgs<double>&, long long, int, cudaStream_t);
template void launch_gather<cplx>(const GatherArgs<cplx>&, long long, int, cudaStream_t);
template void launch_assemble<double>(const AssembleArgs<double>&, int, int, cudaStream_t);
template void launch_assemble<cplx>(const AssembleArgs<cplx>&, int, int, cudaStream_t);
template void launch_apply_pinv<double>(const double*, int, int, const double*, const double*,
                                        const double*, double*, cudaStream_t);
template void launch_apply_pinv<cplx>(const cplx*, int, int, const cplx*, const cplx*, const cplx*,
                                      cplx*, cudaStream_t);
template void launch_tt_random<double>(uint64_t, int, const long long*, const long long*,
                                       double* const*, cudaStream_t);
template void launch_tt_random<cplx>(uint64_t, int, const long long*, const long long*,
                                     cplx* const*, cudaStream_t);

}  // namespace aci
