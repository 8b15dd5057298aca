// Dense contractions of the ACI sweep (FP64 / complex128):
//  * frame half-products (Algorithm 5 before truncation, Eq. (framesrecursive)):
//      LX^n = L^n X^n_l  and  XR^n = X^n_{l+1} R^n, where the frames L^n, R^n are rows I / columns J
//      of the previous half-product: the truncation of Algorithm 5 is a gather on load here;
//  * the Pi block (Eq. (pifromframes)) with f applied in the epilogue (Eq. (localupdate)):
//      Pi = f(LX^1 XR^1, ..., LX^N XR^N), written once, with max|Pi| folded into a running maximum.
// Shapes that depend on ranks chosen on the device are read from the device rank array, so a
// whole sweep can be enqueued without host round trips.
//
// GB300 design. FP64 runs at 2 multiply-adds per clock per SM (1.2 TFLOP/s for the GPU, with
// ~63-cycle latency), so one CTA computing a 32 x 32 tile over K = 256 needs ~60 us: what matters
// is that every SM gets a share of every contraction, including the many small ones of a sweep.
// The live shape is cut into units (32 x 32 output tile, K chunk, product), with enough K chunks
// that the units outnumber the SMs about four to one; a fixed grid of CTAs strides over them and
// writes each unit's partial tile to scratch. The last CTA to finish a tile (a per-tile counter,
// reset by that CTA) sums the tile's partials in a fixed order, applies f and folds the running
// maximum, so the result does not depend on the order in which CTAs finish.
#include "aci_internal.h"

namespace aci {

namespace {

constexpr int BM = 32, BN = 32, BK = 16, NT = 256;
constexpr int TM = 2, TN = 2;  // per-thread outputs; 16 x 16 threads
constexpr int kMinKChunk = 8;

template <class T>
__device__ __forceinline__ T ld_or_zero(const T* p, bool ok) {
    return ok ? *p : s_zero(T());
}
// Loads of other CTAs' partial tiles go through L2.
__device__ __forceinline__ double ldcg_t(const double* p) { return __ldcg(p); }
__device__ __forceinline__ cplx ldcg_t(const cplx* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return mkc(v.x, v.y);
}

struct Plan {
    int M[kMaxInputs], N[kMaxInputs], K[kMaxInputs];
    int tiles[kMaxInputs];  // output tiles per product (combine: one shared output)
    int kc;                 // K chunks per product
    int units;
    int nout;               // outputs (combine: 1)
};

template <class T>
__device__ __forceinline__ Plan make_plan(const GemmArgs<T>& g) {
    Plan pl;
    const int nq = g.nprod;
    int maxkc = 1, tiles_total = 0;
    for (int q = 0; q < kMaxInputs; ++q) {
        pl.M[q] = pl.N[q] = pl.K[q] = 0;
        pl.tiles[q] = 0;
    }
    pl.nout = g.combine ? 1 : nq;
    for (int q = 0; q < nq; ++q) {
        const int z = g.combine ? 0 : q;
        pl.M[q] = dimv(g.M[z], g.chi);
        pl.N[q] = dimv(g.N[z], g.chi);
        pl.K[q] = dimv(g.K[q], g.chi);
        const int kc = (pl.K[q] + kMinKChunk - 1) / kMinKChunk;
        maxkc = kc > maxkc ? kc : maxkc;
    }
    for (int o = 0; o < pl.nout; ++o) {
        pl.tiles[o] = ((pl.M[o] + BM - 1) / BM) * ((pl.N[o] + BN - 1) / BN);
        tiles_total += pl.tiles[o];
    }
    const int per_kc = g.combine ? tiles_total * nq : tiles_total;
    int kc = (g.target_units + per_kc - 1) / (per_kc > 0 ? per_kc : 1);
    kc = kc < 1 ? 1 : (kc > maxkc ? maxkc : kc);
    pl.kc = kc;
    pl.units = per_kc * kc;
    return pl;
}

template <class T>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs<T> g) {
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    __shared__ int s_last;
    // programmatic dependent launch: wait for the previous kernel of the stream before reading
    // anything (the plan reads the device-resolved ranks), then let the next one start launching
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const Plan pl = make_plan(g);
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int nq = g.nprod;

    if (g.flops && blockIdx.x == 0 && tid == 0) {
        const double per = (sizeof(T) == sizeof(cplx)) ? 8.0 : 2.0;
        double f = 0.0;
        for (int q = 0; q < nq; ++q) f += per * (double)pl.M[q] * (double)pl.N[q] * (double)pl.K[q];
        atomicAdd(g.flops, f);
    }

    for (int u = blockIdx.x; u < pl.units; u += gridDim.x) {
        // decode the unit: (output o, tile t, product q, K chunk c); tile_base / unit_base: the
        // tiles and units of the outputs before o
        int o, t, q, c, tile_base = 0, unit_base = 0;
        if (g.combine) {
            o = 0;
            t = u % pl.tiles[0];
            const int rest = u / pl.tiles[0];
            c = rest % pl.kc;
            q = rest / pl.kc;
        } else {
            o = 0;
            while (o + 1 < pl.nout && u - unit_base >= pl.tiles[o] * pl.kc) {
                unit_base += pl.tiles[o] * pl.kc;
                tile_base += pl.tiles[o];
                ++o;
            }
            const int uu = u - unit_base;
            t = uu % pl.tiles[o];
            c = uu / pl.tiles[o];
            q = o;
        }
        const int M = pl.M[o], N = pl.N[o], K = pl.K[q];
        const int tcols = (N + BN - 1) / BN;
        const int m0 = (t / tcols) * BM, n0 = (t % tcols) * BN;
        const int ka = (int)(((long long)K * c) / pl.kc), kb = (int)(((long long)K * (c + 1)) / pl.kc);
        const T* A = g.A[q];
        const T* B = g.B[q];
        const int lda = dimv(g.lda[q], g.chi);
        const int ldb = dimv(g.ldb[q], g.chi);

        T acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = s_zero(T());
        for (int k0 = ka; k0 < kb; k0 += BK) {
            for (int e = tid; e < BM * BK; e += NT) {
                const int i = e / BK, kk = e % BK;
                const int gr = m0 + i, gk = k0 + kk;
                const bool ok = gr < M && gk < kb;
                int src = 0;
                if (ok) src = g.arow ? g.arow[gr] : gr;
                As[kk][i] = ld_or_zero(A + (size_t)src * lda + gk, ok);
            }
            for (int e = tid; e < BK * BN; e += NT) {
                const int kk = e / BN, j = e % BN;
                const int gk = k0 + kk, gc = n0 + j;
                const bool ok = gk < kb && gc < N;
                int col = 0;
                if (ok) col = g.bcol ? g.bcol[gc] : gc;
                Bs[kk][j] = ld_or_zero(B + (size_t)gk * ldb + col, ok);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                T a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = s_fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
        // partial tile -> scratch slot (q, c, t) of output o
        const int tile_id = tile_base + t;
        const int slot = g.combine ? (q * pl.kc + c) * pl.tiles[0] + t : unit_base + c * pl.tiles[o] + t;
        T* part = g.part + (size_t)slot * (BM * BN);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) part[(ty * TM + i) * BN + tx * TN + j] = acc[i][j];
        __threadfence();
        __syncthreads();
        const int expected = g.combine ? pl.kc * nq : pl.kc;
        if (tid == 0) s_last = (atomicAdd(g.tile_count + tile_id, 1) == expected - 1);
        __syncthreads();
        if (!s_last) continue;
        __threadfence();
        // the last CTA of this tile: fixed-order sum of the partials, f, store, running max
        unsigned long long mk = 0;
        T* C = g.C[o];
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int lr = ty * TM + i, gr = m0 + lr;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int lc = tx * TN + j, gc = n0 + lc;
                T v;
                if (g.combine) {
                    T s[kMaxInputs];
                    for (int qq = 0; qq < nq; ++qq) {
                        s[qq] = s_zero(T());
                        for (int cc = 0; cc < pl.kc; ++cc)
                            s[qq] = s_add(s[qq], ldcg_t(g.part + (size_t)((qq * pl.kc + cc) * pl.tiles[0] + t) * (BM * BN) +
                                                             lr * BN + lc));
                    }
                    v = apply_fn(g.op, s, nq);
                } else {
                    v = s_zero(T());
                    for (int cc = 0; cc < pl.kc; ++cc) {
                        const int sl = unit_base + cc * pl.tiles[o] + t;
                        v = s_add(v, ldcg_t(g.part + (size_t)sl * (BM * BN) + lr * BN + lc));
                    }
                }
                if (gr < M && gc < N) {
                    C[(size_t)gr * N + gc] = v;
                    const unsigned long long k = key_of(v);
                    mk = k > mk ? k : mk;  // NaN bits sort above +inf
                }
            }
        }
        if (tid == 0) g.tile_count[tile_id] = 0;  // ready for the next launch
        if (g.smax) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long ov = __shfl_xor_sync(0xffffffffu, mk, off);
                mk = ov > mk ? ov : mk;
            }
            // |v| = key for real, sqrt(key) for complex; sqrt is monotone, so the max commutes with it.
            if ((tid & 31) == 0) {
                const double mag = key_to_mag(__longlong_as_double((long long)mk), T());
                atomicMax(g.smax, (unsigned long long)__double_as_longlong(mag));
            }
        }
    }
}

}  // namespace

int gemm_target_units(int num_sms, int per_sm) { return per_sm * num_sms; }

size_t gemm_part_elems(int Mmax, int Nmax, int nprod, int combine, int num_sms) {
    const size_t tiles = (size_t)((Mmax + BM - 1) / BM) * ((Nmax + BN - 1) / BN);
    const size_t per_kc = combine ? tiles * nprod : tiles * nprod;
    // units < target + per_kc (k chunks are rounded up from target / per_kc); sized for the
    // largest target the split-K tuner may choose
    return (size_t)(gemm_target_units(num_sms, kGemmMaxUnitsPerSm) + per_kc) * BM * BN;
}

size_t gemm_tile_counters(int Mmax, int Nmax, int nprod) {
    return (size_t)((Mmax + BM - 1) / BM) * ((Nmax + BN - 1) / BN) * nprod;
}

template <class T>
void launch_gemm(const GemmArgs<T>& g, int Mmax, int Nmax, cudaStream_t st) {
    if (Mmax <= 0 || Nmax <= 0) return;
    const int grid = 2 * g.num_sms;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = prrlu_pdl_mode();
    cudaLaunchKernelEx(&cfg, gemm_kernel<T>, g);  // errors surface at the sweep's next check
}

template void launch_gemm<double>(const GemmArgs<double>&, int, int, cudaStream_t);
template void launch_gemm<cplx>(const GemmArgs<cplx>&, int, int, cudaStream_t);

}  // namespace aci
