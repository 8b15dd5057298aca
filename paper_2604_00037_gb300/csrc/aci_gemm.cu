// Dense contractions of the ACI sweep (FP64 / complex128):
//  * frame half-products (Algorithm 5 before truncation, Eq. (framesrecursive)):
//      LX^n = L^n X^n_l  and  XR^n = X^n_{l+1} R^n, where the frames L^n, R^n are rows I / columns J
//      of the previous half-product: the truncation of Algorithm 5 is a gather on load here;
//  * the Pi block (Eq. (pifromframes)) with f applied in the epilogue (Eq. (localupdate)):
//      Pi = f(LX^1 XR^1, ..., LX^N XR^N), written once, with max|Pi| folded into a running maximum.
// Shapes that depend on ranks chosen on the device are read from the device rank array, so a
// whole sweep can be enqueued without host round trips; CTAs outside the live shape exit.
//
// GB300 runs FP64 at about 2 FMA/clk/SM (measured 1.2 TFLOP/s for the whole GPU), so these
// kernels are bound by the FP64 pipe, not by memory: what matters is that every SM gets work.
// The tile is 32 x 32 with 256 threads (2 x 2 outputs each, per product).
#include "aci_internal.h"

namespace aci {

namespace {

constexpr int BM = 32, BN = 32, BK = 16, NT = 256;
constexpr int TM = 2, TN = 2;  // per-thread outputs; 16 x 16 threads

template <class T>
__device__ __forceinline__ T ld_or_zero(const T* p, bool ok) {
    return ok ? *p : s_zero(T());
}

template <class T>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs<T> g) {
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int* chi = g.chi;
    const int z = g.combine ? 0 : blockIdx.z;
    const int M = dimv(g.M[z], chi);
    const int N = dimv(g.N[z], chi);
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= M || n0 >= N) return;
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int nprod = g.combine ? g.nprod : 1;

    T acc[2][TM][TN];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[q][i][j] = s_zero(T());

    for (int q = 0; q < nprod; ++q) {
        const int pz = g.combine ? q : z;
        const T* A = g.A[pz];
        const T* B = g.B[pz];
        const int K = dimv(g.K[pz], chi);
        const int lda = dimv(g.lda[pz], chi);
        const int ldb = dimv(g.ldb[pz], chi);
        for (int k0 = 0; k0 < K; k0 += BK) {
            // A tile: BM rows x BK columns, rows optionally gathered.
            for (int e = tid; e < BM * BK; e += NT) {
                const int i = e / BK, kk = e % BK;
                const int gr = m0 + i, gk = k0 + kk;
                const bool ok = gr < M && gk < K;
                int src = 0;
                if (ok) src = g.arow ? g.arow[gr] : gr;
                As[kk][i] = ld_or_zero(A + (size_t)src * lda + gk, ok);
            }
            // B tile: BK rows x BN columns, columns optionally gathered.
            for (int e = tid; e < BK * BN; e += NT) {
                const int kk = e / BN, j = e % BN;
                const int gk = k0 + kk, gc = n0 + j;
                const bool ok = gk < K && gc < N;
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
                    for (int j = 0; j < TN; ++j) acc[q][i][j] = s_fma(a[i], b[j], acc[q][i][j]);
            }
            __syncthreads();
        }
    }

    if (g.flops && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        const double per = (sizeof(T) == sizeof(cplx)) ? 8.0 : 2.0;
        double f = 0.0;
        for (int q = 0; q < nprod; ++q) {
            const int pz = g.combine ? q : z;
            f += per * (double)M * (double)N * (double)dimv(g.K[pz], chi);
        }
        atomicAdd(g.flops, f);
    }

    // Epilogue: f over the products (combine) or a plain store (batch); running max |C|,
    // taken on key bits (integer max) and turned into a magnitude once per warp.
    unsigned long long mk = 0;
    T* C = g.C[z];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int gr = m0 + ty * TM + i;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int gc = n0 + tx * TN + j;
            if (gr < M && gc < N) {
                T v = g.combine ? apply_f(g.op, acc[0][i][j], acc[1][i][j]) : acc[0][i][j];
                C[(size_t)gr * N + gc] = v;
                const unsigned long long k = key_of(v);
                mk = k > mk ? k : mk;  // NaN bits sort above +inf
            }
        }
    }
    if (g.smax) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, mk, off);
            mk = o > mk ? o : mk;
        }
        // |v| = key for real, sqrt(key) for complex; sqrt is monotone, so the max commutes with it.
        if ((tid & 31) == 0) {
            const double mag = key_to_mag(__longlong_as_double((long long)mk), T());
            atomicMax(g.smax, (unsigned long long)__double_as_longlong(mag));
        }
    }
}

}  // namespace

template <class T>
void launch_gemm(const GemmArgs<T>& g, int Mmax, int Nmax, cudaStream_t st) {
    if (Mmax <= 0 || Nmax <= 0) return;
    dim3 grid((Nmax + BN - 1) / BN, (Mmax + BM - 1) / BM, g.combine ? 1 : g.nprod);
    gemm_kernel<T><<<grid, NT, 0, st>>>(g);
}

template void launch_gemm<double>(const GemmArgs<double>&, int, int, cudaStream_t);
template void launch_gemm<cplx>(const GemmArgs<cplx>&, int, int, cudaStream_t);

}  // namespace aci
