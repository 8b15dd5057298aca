// Rank-revealing LU with full pivot search (Algorithm 2, "LDU"), FP64 / complex128.
//
// Each step p takes the entry of largest magnitude among the rows and columns not yet
// pivoted (ties: lowest row * n + col), stops before accepting it when p == chi_hat or
// (p >= 1 and |pivot| <= tau), and otherwise eliminates it with a Schur-complement update
// S <- S - (S[:, j] / S[i, j]) S[i, :] on the unused rows and columns. Instead of the
// paper's in-place row and column swaps, used rows and columns are masked: the pivots,
// D, L and U are the same (L and U are stored in original row / column order).
//
// GB300 design: one cooperative launch per factorisation. CTA g owns a contiguous block of
// columns, kept column-major in a scratch copy W (L2-resident). Every step has exactly one
// grid-wide synchronisation, carried by the data itself: each CTA publishes its best
// candidate (value and position) and that candidate's whole column in a record tagged with
// the step number (release store); every CTA then waits for the G tags of the step (acquire
// loads, bounded spin), picks the same winner, and reads the winner's column for its own
// update. Records and columns are double-buffered by step parity, so no CTA can overwrite
// a record another CTA has not read yet (it would first need that CTA's next record).
// The Schur update of step p is fused with the local argmax of step p+1.
#include <climits>

#include "aci_internal.h"

namespace aci {

namespace {

constexpr int PT = 256;
constexpr int NWARP = PT / 32;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Loads of data written by other CTAs during this launch go through L2 (never a stale L1 line).
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ cplx ldcg(const cplx* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return mkc(v.x, v.y);
}
__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }

__device__ __forceinline__ bool better(double k1, int l1, double k2, int l2) {
    return k1 > k2 || (k1 == k2 && l1 < l2);
}

// Block-wide (key, linear index) argmax; the result is returned to every thread.
__device__ __forceinline__ void block_argmax(double& key, int& lin, double* skey, int* slin) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double ok = __shfl_xor_sync(0xffffffffu, key, off);
        const int ol = __shfl_xor_sync(0xffffffffu, lin, off);
        if (better(ok, ol, key, lin)) { key = ok; lin = ol; }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) { skey[warp] = key; slin[warp] = lin; }
    __syncthreads();
    if (warp == 0) {
        key = lane < NWARP ? skey[lane] : -2.0;
        lin = lane < NWARP ? slin[lane] : INT_MAX;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ok = __shfl_xor_sync(0xffffffffu, key, off);
            const int ol = __shfl_xor_sync(0xffffffffu, lin, off);
            if (better(ok, ol, key, lin)) { key = ok; lin = ol; }
        }
        if (lane == 0) { skey[NWARP] = key; slin[NWARP] = lin; }
    }
    __syncthreads();
    key = skey[NWARP];
    lin = slin[NWARP];
}

__device__ __forceinline__ void set_val(PivRec* r, double v) { r->vre = v; r->vim = 0.0; }
__device__ __forceinline__ void set_val(PivRec* r, cplx v) { r->vre = v.re; r->vim = v.im; }
__device__ __forceinline__ void get_val(const PivRec* r, double& v) { v = __ldcg(&r->vre); }
__device__ __forceinline__ void get_val(const PivRec* r, cplx& v) { v = mkc(__ldcg(&r->vre), __ldcg(&r->vim)); }

__device__ __forceinline__ double sanitize_key(double k) { return (k != k) ? INFINITY : k; }

template <class T>
__global__ void __launch_bounds__(PT) prrlu_kernel(PrrluArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    const int m = dimv(a.m, a.chi), n = dimv(a.n, a.chi);
    const int c0 = (int)(((long long)n * g) / G), c1 = (int)(((long long)n * (g + 1)) / G);
    const int w = c1 - c0;
    const int wmax = (a.nmax + G - 1) / G;
    const int mmax = a.mmax;

    T* lcol = reinterpret_cast<T*>(smem_raw);           // [mmax] multipliers S[r, j] / pivot
    T* prow = lcol + mmax;                               // [wmax] pivot row, own columns
    double* skey = reinterpret_cast<double*>(prow + wmax);  // [NWARP + 1]
    int* slin = reinterpret_cast<int*>(skey + NWARP + 1);   // [NWARP + 1]
    int* sint = slin + NWARP + 1;                           // [4] flags
    unsigned char* rowused = reinterpret_cast<unsigned char*>(sint + 4);  // [mmax]
    unsigned char* colused = rowused + mmax;                              // [wmax]

    T* Wb = a.W + (size_t)c0 * mmax;

    for (int e = tid; e < m * w; e += PT) {
        const int r = e / w, cc = e % w;
        Wb[(size_t)cc * mmax + r] = a.Min[(size_t)r * n + c0 + cc];
    }
    for (int r = tid; r < m; r += PT) rowused[r] = 0;
    for (int cc = tid; cc < w; cc += PT) colused[cc] = 0;
    if (tid < 4) sint[tid] = 0;
    __syncthreads();

    const int kmax = min(min(m, n), a.chimax);
    const double S = a.rel ? __longlong_as_double((long long)*a.smax) : 0.0;
    const double tau = a.rel ? a.tol * S : a.tol;

    double bkey = -1.0;
    int blin = INT_MAX;
    for (int e = tid; e < m * w; e += PT) {
        const int cc = e / m, r = e - cc * m;
        const double k = sanitize_key(s_key(Wb[(size_t)cc * mmax + r]));
        const int lin = r * n + c0 + cc;
        if (better(k, lin, bkey, blin)) { bkey = k; blin = lin; }
    }

    int p = 0;
    double eps = 0.0;
    for (;;) {
        block_argmax(bkey, blin, skey, slin);
        const int buf = p & 1;
        PivRec* myrec = a.rec + (size_t)buf * G + g;
        T* myslot = a.slots + ((size_t)buf * G + g) * mmax;
        if (blin != INT_MAX) {
            const int cc = (blin % n) - c0;
            for (int r = tid; r < m; r += PT) myslot[r] = Wb[(size_t)cc * mmax + r];
        }
        __syncthreads();
        const unsigned long long tag = (a.epoch << 24) | (unsigned long long)(p + 1);
        if (tid == 0) {
            if (blin != INT_MAX) {
                const int r = blin / n, c = blin % n;
                myrec->key = bkey;
                set_val(myrec, Wb[(size_t)(c - c0) * mmax + r]);
                myrec->r = r;
                myrec->c = c;
            } else {
                myrec->key = -1.0;
                set_val(myrec, s_zero(T()));
                myrec->r = -1;
                myrec->c = -1;
            }
            __threadfence();
            st_release_u64(&myrec->tag, tag);
        }
        // One grid-wide synchronisation per step: wait for the G records of this step.
        if (tid < G) {
            const PivRec* rr = a.rec + (size_t)buf * G + tid;
            long long spins = 0;
            while (ld_acquire_u64(&rr->tag) != tag) {
                if (++spins > kSpinLimit) {
                    atomicOr(a.err, DEVERR_TIMEOUT);
                    sint[0] = 1;
                    break;
                }
            }
        }
        __threadfence();
        __syncthreads();
        if (sint[0]) return;  // gave up waiting; the host reads ACI_E_TIMEOUT

        double wkey = -1.0;
        int wlin = INT_MAX;
        if (tid < G) {
            const PivRec* rr = a.rec + (size_t)buf * G + tid;
            const int r = ldcg(&rr->r);
            if (r >= 0) {
                wkey = __ldcg(&rr->key);
                wlin = r * n + ldcg(&rr->c);
            }
        }
        const int mylin = wlin;
        block_argmax(wkey, wlin, skey, slin);
        if (tid < G && mylin == wlin && wlin != INT_MAX) sint[1] = tid;
        __syncthreads();
        if (wlin == INT_MAX) {  // no unused entry is left
            eps = 0.0;
            break;
        }
        const double mag = key_to_mag(wkey, T());
        if (!(wkey < INFINITY)) {
            if (g == 0 && tid == 0) atomicOr(a.err, DEVERR_NUMERIC);
            eps = mag;
            break;
        }
        if (p == kmax || (p >= 1 && mag <= tau)) {
            eps = mag;
            break;
        }
        const int wi = sint[1];
        const PivRec* wr = a.rec + (size_t)buf * G + wi;
        T piv;
        get_val(wr, piv);
        const int ri = wlin / n, cj = wlin % n;
        const bool zpiv = s_iszero(piv);
        if (g == 0 && tid == 0) {
            a.piv_rows[p] = ri;
            a.piv_cols[p] = cj;
            a.D[p] = piv;
        }
        const T* wslot = a.slots + ((size_t)buf * G + wi) * mmax;
        for (int r = tid; r < m; r += PT) {
            T l = s_zero(T());
            if (!rowused[r] && r != ri && !zpiv) l = s_div(ldcg(wslot + r), piv);
            lcol[r] = l;
        }
        if (a.L) {  // column p of L, rows split across the CTAs
            const int r0 = (int)(((long long)m * g) / G), r1 = (int)(((long long)m * (g + 1)) / G);
            for (int r = r0 + tid; r < r1; r += PT) {
                T v;
                if (r == ri) v = s_one(T());
                else if (rowused[r] || zpiv) v = s_zero(T());
                else v = s_div(ldcg(wslot + r), piv);
                a.L[(size_t)p * a.Lld + r] = v;
            }
        }
        for (int cc = tid; cc < w; cc += PT) {
            const T v = Wb[(size_t)cc * mmax + ri];
            prow[cc] = v;
            if (a.U) {
                const int c = c0 + cc;
                T u;
                if (c == cj) u = s_one(T());
                else if (colused[cc] || zpiv) u = s_zero(T());
                else u = s_div(v, piv);
                a.U[(size_t)p * a.Uld + c] = u;
            }
        }
        __syncthreads();
        if (tid == 0) {
            rowused[ri] = 1;
            if (cj >= c0 && cj < c1) colused[cj - c0] = 1;
        }
        __syncthreads();
        // Schur-complement update of the unused block, fused with the next local argmax.
        bkey = -1.0;
        blin = INT_MAX;
        for (int e = tid; e < m * w; e += PT) {
            const int cc = e / m, r = e - cc * m;
            if (rowused[r] | colused[cc]) continue;
            T* ptr = Wb + (size_t)cc * mmax + r;
            const T v = s_fms(lcol[r], prow[cc], *ptr);
            *ptr = v;
            const double k = sanitize_key(s_key(v));
            const int lin = r * n + c0 + cc;
            if (better(k, lin, bkey, blin)) { bkey = k; blin = lin; }
        }
        ++p;
    }
    if (g == 0 && tid == 0) {
        if (a.flops) {  // Schur-update multiply-adds: sum_{q<p} (m-q-1)(n-q-1)
            const double per = (sizeof(T) == sizeof(cplx)) ? 8.0 : 2.0;
            double f = 0.0;
            for (int q = 0; q < p; ++q) f += (double)(m - q - 1) * (double)(n - q - 1);
            atomicAdd(a.flops, per * f);
        }
        *a.eps_out = eps;
        if (a.k_out) *a.k_out = p;
        if (a.out_chi_idx >= 0) const_cast<int*>(a.chi)[a.out_chi_idx] = p;
    }
}

}  // namespace

int prrlu_grid(int nmax, int num_sms) {
    int G = nmax / 4;
    if (G < 1) G = 1;
    if (G > num_sms) G = num_sms;
    if (G > PT) G = PT;  // one waiting thread per record
    return G;
}

template <class T>
size_t prrlu_smem_bytes(int mmax, int nmax, int G) {
    const int wmax = (nmax + G - 1) / G;
    size_t b = sizeof(T) * (size_t)(mmax + wmax);
    b += sizeof(double) * (NWARP + 1) + sizeof(int) * (NWARP + 1) + sizeof(int) * 4;
    b += (size_t)mmax + (size_t)wmax;
    return (b + 15) & ~(size_t)15;
}

template <class T>
cudaError_t launch_prrlu(const PrrluArgs<T>& a, int G, cudaStream_t st) {
    const size_t smem = prrlu_smem_bytes<T>(a.mmax, a.nmax, G);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(prrlu_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    PrrluArgs<T> copy = a;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)prrlu_kernel<T>, dim3(G), dim3(PT), args, smem, st);
}

template cudaError_t launch_prrlu<double>(const PrrluArgs<double>&, int, cudaStream_t);
template cudaError_t launch_prrlu<cplx>(const PrrluArgs<cplx>&, int, cudaStream_t);
template size_t prrlu_smem_bytes<double>(int, int, int);
template size_t prrlu_smem_bytes<cplx>(int, int, int);

}  // namespace aci
