// Rank-revealing LU with full pivot search (Algorithm 2, "LDU"), FP64 / complex128.
//
// Each step p takes the entry of largest magnitude among the rows and columns not yet
// pivoted (ties: lowest row * n + col), stops before accepting it when p == chi_hat or
// (p >= 1 and |pivot| <= tau), and otherwise eliminates it with a Schur-complement update
// S <- S - (S[:, j] / S[i, j]) S[i, :] on the unused rows and columns. Instead of the
// paper's in-place row and column swaps, used rows and columns are masked: the pivots,
// D, L and U are the same (L and U are stored in original row / column order). The
// multipliers use one reciprocal of the pivot per step.
//
// GB300 design. One cooperative launch per factorisation; the number of CTAs that take part
// is chosen on the device from the live shape (about kEpc entries per CTA, at least one column
// each), so small blocks run in one CTA with no grid-wide synchronisation at all. CTA g owns a
// contiguous block of columns, kept column-major in shared memory when the worst case fits
// (else in an L2-resident global copy). The pivot steps are strictly sequential; each one
// costs one exchange of candidates between CTAs, made of self-validating 8-byte words: the low
// 32 bits carry data, the high 32 bits the step's tag. Every CTA writes its best candidate (key,
// position, value) as such words, then polls the G records of the step; because every 8-byte word
// is written and read atomically and carries its own tag, no fence, acquire or release is needed,
// and a word from an older step can never be mistaken for a current one. After the decision the
// CTA that owns the winning column publishes it the same way and the others read it. Records and
// columns alternate between two buffers by step parity: a CTA can only overwrite a buffer after
// every other CTA has published its next record, which each does only after it has read the
// buffer. The caller clears the exchange area once per sequence of launches and gives each launch
// a distinct tag base.
// The Schur update of step p is fused with the local argmax of step p+1.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstdlib>
#include <mutex>
#include <set>

#include <cooperative_groups.h>

#include "aci_internal.h"

namespace aci {

namespace {

constexpr int PT = 256;
constexpr int NWARP = PT / 32;

template <class T> struct Words;  // 8-byte exchange words per value
template <> struct Words<double> { static constexpr int value = 2; };
template <> struct Words<cplx> { static constexpr int value = 4; };
constexpr int kRecWords = 8;      // key (2), position (1), value (up to 4), spare (1)

__device__ __forceinline__ void st_word(unsigned long long* p, unsigned int data, unsigned int tag) {
    const unsigned long long v = ((unsigned long long)tag << 32) | data;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int word_tag(unsigned long long w) { return (unsigned int)(w >> 32); }
__device__ __forceinline__ double ldcg_val(const double* p) { return __ldcg(p); }
__device__ __forceinline__ cplx ldcg_val(const cplx* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return mkc(v.x, v.y);
}
__device__ __forceinline__ unsigned int word_data(unsigned long long w) { return (unsigned int)w; }

__device__ __forceinline__ void put_double(unsigned long long* p, double v, unsigned int tag) {
    st_word(p, (unsigned int)__double2hiint(v), tag);
    st_word(p + 1, (unsigned int)__double2loint(v), tag);
}
__device__ __forceinline__ void put_val(unsigned long long* p, double v, unsigned int tag) { put_double(p, v, tag); }
__device__ __forceinline__ void put_val(unsigned long long* p, cplx v, unsigned int tag) {
    put_double(p, v.re, tag);
    put_double(p + 2, v.im, tag);
}
__device__ __forceinline__ double dbl_of(unsigned long long hi, unsigned long long lo) {
    return __hiloint2double((int)word_data(hi), (int)word_data(lo));
}
__device__ __forceinline__ void val_of(const unsigned long long* w, double& v) { v = dbl_of(w[0], w[1]); }
__device__ __forceinline__ void val_of(const unsigned long long* w, cplx& v) {
    v = mkc(dbl_of(w[0], w[1]), dbl_of(w[2], w[3]));
}

// Read NW consecutive words once all of them carry `tag`; false after `limit` polls.
template <int NW>
__device__ __forceinline__ bool get_words(const unsigned long long* p, unsigned int tag, unsigned long long* out,
                                          long long limit) {
    long long spins = 0;
    for (;;) {
        bool ok = true;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            out[i] = ld_word(p + i);
            ok &= word_tag(out[i]) == tag;
        }
        if (ok) return true;
        if (++spins > limit) return false;
    }
}

// Programmatic dependent launch: a kernel launched with the programmatic-serialization attribute
// may start while the previous kernel of its stream finishes; it waits here, before reading any
// of that kernel's outputs (a no-op when launched without the attribute).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// ... and lets the next kernel of the stream, if launched so, start its launch (it waits for this
// grid's completion before reading anything): issued after the pivot loop, so that a waiting
// dependent never holds SMs while the search runs.
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Keys are non-negative doubles (|v|, or re^2 + im^2), so they order like their bit patterns:
// the argmax compares 64-bit integers (the FP64 pipe, 2 ops/clk/SM on GB300, is left to the
// Schur update). A NaN key sorts above +inf and surfaces as a numeric error at the stop test.
// (key bits, linear index) = (0, INT_MAX) means "no candidate"; any real entry beats it.
typedef unsigned long long kbits_t;
__device__ __forceinline__ kbits_t key_bits(double k) { return (kbits_t)__double_as_longlong(k); }

// Round a shared-memory pointer up to 16 bytes (matches the padding in the byte counts).
template <class P>
__device__ __forceinline__ P* align16(void* p) {
    return reinterpret_cast<P*>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
}

// The step's decision, taken by one thread and read by all (keeps FP64 work off the others).
template <class T> struct __align__(16) Decision {
    int code;  // 0 = accept the pivot, 1 = stop, 2 = stop on a non-finite pivot
    int zpiv;  // the pivot is exactly zero (all-zero block)
    int lin;   // winner's position and owning CTA (used by the register-resident kernel)
    int gw;
    double eps;
    T inv;     // 1 / pivot (0 when zpiv)
    T piv;
};

// 1/d for a real pivot: the hardware's approximate FP64 reciprocal (PTX rcp.approx.ftz.f64) as
// the seed, then two Newton-Raphson steps r <- r + r (1 - d r) in FP64; each step squares the
// relative error, so a seed good to about 20 bits ends below one ulp (the GPU tests check every
// result against 1/x to two ulp). On this GPU a dependent FP64 operation takes ~63 cycles and a
// correctly rounded division ~570, and the reciprocal sits on the critical path of every pivot
// step. Outside 2^(+-99) (no subnormal seed) the division is used instead.
__device__ __forceinline__ double fast_recip(double d) {
    // range test on the biased exponent (integer work): 2^-99 <= |d| < 2^100
    const unsigned ex = ((unsigned)__double2hiint(d) >> 20) & 0x7FFu;
    if (ex < 1023u - 99u || ex >= 1023u + 100u) return 1.0 / d;
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ double recip_of(double d) { return fast_recip(d); }
// 1/d for a complex pivot: conj(d) / |d|^2 with the real reciprocal above, when both parts are
// within 2^(+-480) (so |d|^2 neither overflows nor loses precision); Smith's division (two FP64
// divisions, ~1100 cycles on the step's critical path) otherwise. Each part is within a few units
// in the last place of the exact reciprocal's.
__device__ __forceinline__ cplx recip_of(cplx d) {
    const unsigned er = ((unsigned)__double2hiint(d.re) >> 20) & 0x7FFu;
    const unsigned ei = ((unsigned)__double2hiint(d.im) >> 20) & 0x7FFu;
    const unsigned e = er > ei ? er : ei;
    if (e < 1023u - 480u || e > 1023u + 480u) return s_div(s_one(cplx()), d);
    const double r = fast_recip(fma(d.re, d.re, d.im * d.im));
    return mkc(d.re * r, -d.im * r);
}

// The stop test |pivot| <= tau as a compare on key bits. Real keys are |v|. A complex key is
// re*re + im*im (each rounded) and |v| is its correctly rounded square root, which is monotone:
// sqrt(key) <= tau exactly when key <= K(tau), the largest double whose root is at most tau. K(tau)
// is found once per launch (a few square roots near tau * tau), so no step takes a square root.
__device__ inline kbits_t tau_key(double tau, double) { return key_bits(tau); }
__device__ inline kbits_t tau_key(double tau, cplx) {
    if (!(tau >= 0.0)) return 0;
    if (isinf(tau)) return key_bits(INFINITY);
    double k = __dmul_rn(tau, tau);
    while (k > 0.0 && __dsqrt_rn(k) > tau) k = nextafter(k, 0.0);
    while (k < DBL_MAX && __dsqrt_rn(nextafter(k, INFINITY)) <= tau) k = nextafter(k, INFINITY);
    return key_bits(k);
}
// K(tau) for every thread of the CTA: thread 0 forms it (complex) and a block barrier shares it.
// Called by all threads of the CTA alike.
template <class T>
__device__ __forceinline__ kbits_t tau_key_cta(double tau) {
    if constexpr (sizeof(T) == sizeof(double)) {
        return key_bits(tau);
    } else {
        __shared__ kbits_t s_tkey;
        if (threadIdx.x == 0) s_tkey = tau_key(tau, T());
        __syncthreads();
        return s_tkey;
    }
}
// pivot == 0 on the bits (both parts +-0), no FP64 compare
__device__ __forceinline__ bool val_is_zero(double v) { return (((unsigned long long)__double_as_longlong(v)) << 1) == 0; }
__device__ __forceinline__ bool val_is_zero(cplx v) {
    return ((((unsigned long long)__double_as_longlong(v.re)) | ((unsigned long long)__double_as_longlong(v.im))) << 1) == 0;
}

// The stop test of Algorithm 2 and the multiplier scale for the step's winner: |pivot| <= tau
// (tkey = tau_key(tau)) and pivot == 0 are decided on bits, and |pivot| (a square root for complex
// values) is formed only at the stop, which keeps FP64 work (~64 cycles per warp-wide operation
// here, in every warp that takes the decision) off the steps.
template <class T>
__device__ __forceinline__ void decide(Decision<T>* d, kbits_t wkey, int wlin, T piv, int p, int kmax, kbits_t tkey,
                                       bool with_inv = true) {
    int code = 0;
    double e = 0.0;
    d->zpiv = 0;
    d->inv = s_zero(T());
    if (wlin == INT_MAX) {
        code = 1;
    } else {
        // pivot == 0 from the key bits where they decide it (real: the key is |pivot|; complex: a
        // nonzero key rules it out), so the common step does not wait for the value's shuffle (in
        // the real path that wait cost 3.5 % of the bench product)
        constexpr bool is_real = sizeof(T) == sizeof(double);
        const bool below = wkey <= tkey;
        const bool zero = is_real ? (wkey == 0) : (wkey == 0 && val_is_zero(piv));
        if (wkey >= key_bits(INFINITY)) {
            code = 2;
            e = key_to_mag(__longlong_as_double((long long)wkey), T());
        } else if (p == kmax || (p >= 1 && below)) {
            code = 1;
            e = key_to_mag(__longlong_as_double((long long)wkey), T());
        } else if (zero) {
            d->zpiv = 1;
        } else if (with_inv) {
            d->inv = recip_of(piv);
        }
    }
    d->code = code;
    d->eps = e;
}
__device__ __forceinline__ bool better(kbits_t k1, int l1, kbits_t k2, int l2) {
    return k1 > k2 || (k1 == k2 && l1 < l2);
}

// Block-wide (key, linear index) argmax; the result is returned to every thread.
__device__ __forceinline__ void block_argmax(kbits_t& key, int& lin, kbits_t* skey, int* slin) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const kbits_t ok = __shfl_xor_sync(0xffffffffu, key, off);
        const int ol = __shfl_xor_sync(0xffffffffu, lin, off);
        if (better(ok, ol, key, lin)) { key = ok; lin = ol; }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) { skey[warp] = key; slin[warp] = lin; }
    __syncthreads();
    if (warp == 0) {
        key = lane < NWARP ? skey[lane] : 0ull;
        lin = lane < NWARP ? slin[lane] : INT_MAX;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const kbits_t ok = __shfl_xor_sync(0xffffffffu, key, off);
            const int ol = __shfl_xor_sync(0xffffffffu, lin, off);
            if (better(ok, ol, key, lin)) { key = ok; lin = ol; }
        }
        if (lane == 0) { skey[NWARP] = key; slin[NWARP] = lin; }
    }
    __syncthreads();
    key = skey[NWARP];
    lin = slin[NWARP];
}

// Multiply-adds of p Schur-complement updates of an m x n block, sum over q < p of
// (m - q - 1)(n - q - 1), in closed form (exact in 64-bit integers for m, n <= 65536, p <= 8192):
// a loop of dependent FP64 additions would sit on the kernel's tail.
__device__ __forceinline__ double schur_mults(int m, int n, int p) {
    const long long a = m - 1, b = n - 1, q = p;
    const long long s1 = q * (q - 1) / 2, s2 = (q - 1) * q * (2 * q - 1) / 6;
    return (double)(q * a * b - (a + b) * s1 + s2);
}

__host__ __device__ inline int live_ctas(long long mn, int n, int G, int epc) {
    long long g = (mn + epc - 1) / epc;
    if (g < 1) g = 1;
    if (g > G) g = G;
    if (g > n) g = n;
    return (int)g;
}

// The live block is the single-CTA kernel's (see PrrluArgs::small_*).
template <class T>
__device__ __forceinline__ bool small_block(const PrrluArgs<T>& a, int m, int n) {
    return a.small_elems > 0 && m <= a.small_m && n <= a.small_n && (long long)m * n <= a.small_elems;
}

template <class T, bool SMEMW>
__global__ void __launch_bounds__(PT) prrlu_kernel(PrrluArgs<T> a) {
    grid_dependency_wait();  // launched early behind the previous kernel of the stream: its outputs are read below
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int WPV = Words<T>::value;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    const int m = dimv(a.m, a.chi), n = dimv(a.n, a.chi);
    if (small_block(a, m, n)) return;  // the single-CTA kernel's block
    const long long spin_limit = a.spin_limit > 0 ? a.spin_limit : kSpinLimit;
    const int Ge = live_ctas((long long)m * n, n, G, a.epc);
    if (g >= Ge) return;
    const int c0 = (int)(((long long)n * g) / Ge), c1 = (int)(((long long)n * (g + 1)) / Ge);
    const int w = c1 - c0;
    const int mmax = a.mmax;

    // shared memory: [W block] lcol[mmax] prow[wcols] sval[G] | skey slin sint | rowused colused
    T* Wsm = reinterpret_cast<T*>(smem_raw);
    T* lcol = Wsm + (SMEMW ? a.wcap_elems : 0);
    T* prow = lcol + mmax;
    T* sval = prow + a.wcap_cols;
    Decision<T>* dec = align16<Decision<T>>(sval + G);
    kbits_t* skey = reinterpret_cast<kbits_t*>(dec + 1);
    int* slin = reinterpret_cast<int*>(skey + NWARP + 1);
    int* sint = slin + NWARP + 1;
    unsigned char* rowused = reinterpret_cast<unsigned char*>(sint + 4);
    unsigned char* colused = rowused + mmax;

    T* Wb;
    int ldw;
    if (SMEMW) {
        Wb = Wsm;
        ldw = m;
    } else {
        Wb = a.W + (size_t)c0 * mmax;
        ldw = mmax;
    }
    unsigned long long* recs = a.ll;                                  // [2][G][kRecWords]
    unsigned long long* cols = a.ll + 2 * (size_t)G * kRecWords;      // [2][G][mmax * WPV]

    // Copy the own column block (thread = row) and find the first local candidate.
    kbits_t bkey = 0;
    int blin = INT_MAX;
    for (int r = tid; r < m; r += PT) {
        rowused[r] = 0;
        const T* src = a.Min + (size_t)r * n + c0;
        const int rn = r * n + c0;
        for (int cc = 0; cc < w; ++cc) {
            const T v = src[cc];
            Wb[(size_t)cc * ldw + r] = v;
            const kbits_t k = key_of(v);
            if (better(k, rn + cc, bkey, blin)) { bkey = k; blin = rn + cc; }
        }
    }
    for (int cc = tid; cc < w; cc += PT) colused[cc] = 0;
    if (tid < 4) sint[tid] = 0;
    __syncthreads();

    const int kmax = min(min(m, n), a.chimax);
    const double S = a.rel ? __longlong_as_double((long long)*a.smax) : 0.0;
    const double tau = a.rel ? a.tol * S : a.tol;
    const kbits_t tkey = threadIdx.x == 0 ? tau_key(tau, T()) : 0;  // thread 0 takes the decision

    int p = 0;
    double eps = 0.0;
    for (;;) {
        block_argmax(bkey, blin, skey, slin);
        const unsigned int tag = a.tagbase + (unsigned int)(p + 1);
        const int buf = p & 1;
        kbits_t wkey = bkey;
        int wlin = blin;
        T piv = s_zero(T());
        int gw = g;  // CTA that owns the winning column
        if (Ge == 1) {
            if (wlin != INT_MAX) piv = Wb[(size_t)(wlin % n - c0) * ldw + wlin / n];
        } else {
            // publish: candidate column and record, as tagged words (no fence needed)
            unsigned long long* myrec = recs + ((size_t)buf * G + g) * kRecWords;
            // the column itself is published by the winner's owner, after the decision
            if (tid == 0) {
                st_word(myrec, (unsigned int)(bkey >> 32), tag);
                st_word(myrec + 1, (unsigned int)bkey, tag);
                st_word(myrec + 2, (unsigned int)blin, tag);
                T v = s_zero(T());
                if (blin != INT_MAX) v = Wb[(size_t)(blin % n - c0) * ldw + blin / n];
                put_val(myrec + 3, v, tag);
            }
            // gather the Ge records of this step (one poller per record)
            wkey = 0;
            wlin = INT_MAX;
            if (tid < Ge) {
                unsigned long long rw[3 + WPV];
                if (!get_words<3 + WPV>(recs + ((size_t)buf * G + tid) * kRecWords, tag, rw, spin_limit)) {
                    atomicOr(a.err, DEVERR_TIMEOUT);
                    sint[0] = 1;
                } else {
                    wkey = ((kbits_t)word_data(rw[0]) << 32) | word_data(rw[1]);
                    wlin = (int)word_data(rw[2]);
                    T v;
                    val_of(rw + 3, v);
                    sval[tid] = v;
                }
            }
            block_argmax(wkey, wlin, skey, slin);
            if (sint[0]) return;  // gave up waiting; the host reads ACI_E_TIMEOUT
            if (wlin != INT_MAX) {
                const int cj = wlin % n;
                gw = (int)((((long long)cj + 1) * Ge - 1) / n);
                piv = sval[gw];
            }
        }
        if (tid == 0) decide(dec, wkey, wlin, piv, p, kmax, tkey);
        __syncthreads();
        if (dec->code) {  // stop: no unused entry left, tolerance or rank cap reached, or non-finite
            if (dec->code == 2 && g == 0 && tid == 0) atomicOr(a.err, DEVERR_NUMERIC);
            eps = dec->eps;
            break;
        }
        const int ri = wlin / n, cj = wlin % n;
        const bool zpiv = dec->zpiv;
        const T inv = dec->inv;
        if (g == 0 && tid == 0) {
            a.piv_rows[p] = ri;
            a.piv_cols[p] = cj;
            a.D[p] = piv;
        }
        // Multipliers S[r, cj] / pivot from the winning column; pivot row of the own columns.
        // Row ri and column cj become used here; the loops below never read those flags for them.
        // Only the winning column's owner publishes it (tagged words, read by the other CTAs): one
        // column per step crosses L2 instead of every CTA's candidate column.
        if (Ge == 1 || g == gw) {
            const T* colp = Wb + (size_t)(cj - c0) * ldw;
            unsigned long long* oc = cols + ((size_t)buf * G + g) * (size_t)mmax * WPV;
            for (int r = tid; r < m; r += PT) {
                const T v = colp[r];
                if (Ge > 1) put_val(oc + (size_t)r * WPV, v, tag);
                lcol[r] = (rowused[r] || r == ri || zpiv) ? s_zero(T()) : s_mul(v, inv);
            }
        } else {
            const unsigned long long* wc = cols + ((size_t)buf * G + gw) * (size_t)mmax * WPV;
            for (int r = tid; r < m; r += PT) {
                unsigned long long cw[WPV];
                if (!get_words<WPV>(wc + (size_t)r * WPV, tag, cw, spin_limit)) {
                    atomicOr(a.err, DEVERR_TIMEOUT);
                    sint[1] = 1;
                    break;
                }
                T v;
                val_of(cw, v);
                lcol[r] = (rowused[r] || r == ri || zpiv) ? s_zero(T()) : s_mul(v, inv);
            }
        }
        for (int cc = tid; cc < w; cc += PT) {
            const T v = Wb[(size_t)cc * ldw + ri];
            prow[cc] = v;
            if (a.U) {
                const int c = c0 + cc;
                T u;
                if (c == cj) u = s_one(T());
                else if (colused[cc] || zpiv) u = s_zero(T());
                else u = s_mul(v, inv);
                a.U[(size_t)p * a.Uld + c] = u;
            }
        }
        __syncthreads();
        if (sint[1]) return;
        if (tid == 0) {
            rowused[ri] = 1;
            if (cj >= c0 && cj < c1) colused[cj - c0] = 1;
        }
        if (a.L) {  // column p of L, rows split across the CTAs
            const int r0 = (int)(((long long)m * g) / Ge), r1 = (int)(((long long)m * (g + 1)) / Ge);
            for (int r = r0 + tid; r < r1; r += PT) a.L[(size_t)p * a.Lld + r] = (r == ri) ? s_one(T()) : lcol[r];
        }
        __syncthreads();
        // Schur-complement update of the unused block (thread = row), fused with the next
        // local argmax.
        bkey = 0;
        blin = INT_MAX;
        for (int r = tid; r < m; r += PT) {
            if (rowused[r]) continue;
            const T l = lcol[r];
            const int rn = r * n + c0;
            T* rowp = Wb + r;
            for (int cc = 0; cc < w; ++cc) {
                if (colused[cc]) continue;
                T* ptr = rowp + (size_t)cc * ldw;
                const T v = s_fms(l, prow[cc], *ptr);
                *ptr = v;
                const kbits_t k = key_of(v);
                if (better(k, rn + cc, bkey, blin)) { bkey = k; blin = rn + cc; }
            }
        }
        ++p;
    }
    if (g == 0 && tid == 0) {
        if (a.flops) {  // Schur-update multiply-adds: sum_{q<p} (m-q-1)(n-q-1)
            const double per = (sizeof(T) == sizeof(cplx)) ? 8.0 : 2.0;
            const double f = schur_mults(m, n, p);
            atomicAdd(a.flops, per * f);
        }
        *a.eps_out = eps;
        if (a.k_out) *a.k_out = p;
        if (a.out_chi_idx >= 0) const_cast<int*>(a.chi)[a.out_chi_idx] = p;
    }
}

// ---------------------------------------------------------------- cluster variant
// For blocks that 16 SMs of FP64 can update fast enough (the usual case), the CTAs of one
// thread-block cluster share the work and exchange through distributed shared memory: every
// step, each CTA writes its best candidate into every CTA's candidate slots, one hardware
// cluster barrier (release/acquire) follows, each CTA reduces the C candidates locally, and
// reads the winning column straight out of the owner's shared memory (a pivot column is never
// written again once chosen). No L2 round trip and no software spin is on the step's path.
template <class T> struct __align__(16) Cand {
    kbits_t key;
    int lin;
    int pad;
    T val;
};

template <class T, bool SMEMW>
__global__ void __launch_bounds__(PT) prrlu_cluster_kernel(PrrluArgs<T> a) {
    grid_dependency_wait();  // launched early behind the previous kernel of the stream: its outputs are read below
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int g = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = dimv(a.m, a.chi), n = dimv(a.n, a.chi);
    if (small_block(a, m, n)) return;  // every CTA of the cluster returns before any exchange
    const int c0 = (int)(((long long)n * g) / C), c1 = (int)(((long long)n * (g + 1)) / C);
    const int w = c1 - c0;
    const int mmax = a.mmax;

    // shared memory: [W block] lcol[mmax] prow[wcols] cand[2][C] | wbest | rowused colused
    T* Wsm = reinterpret_cast<T*>(smem_raw);
    T* lcol = Wsm + (SMEMW ? a.wcap_elems : 0);
    T* prow = lcol + mmax;
    Cand<T>* cand = align16<Cand<T>>(prow + a.wcap_cols);            // [2][C]
    Cand<T>* wbest = cand + 2 * C;                                    // [NWARP + 1]
    Decision<T>* dec = reinterpret_cast<Decision<T>*>(wbest + NWARP + 1);
    unsigned char* rowused = reinterpret_cast<unsigned char*>(dec + 1);
    unsigned char* colused = rowused + mmax;

    T* Wb;
    int ldw;
    if (SMEMW) {
        Wb = Wsm;
        ldw = m;
    } else {
        Wb = a.W + (size_t)c0 * mmax;
        ldw = mmax;
    }

    kbits_t bkey = 0;
    int blin = INT_MAX;
    for (int r = tid; r < m; r += PT) {
        rowused[r] = 0;
        const T* src = a.Min + (size_t)r * n + c0;
        const int rn = r * n + c0;
        for (int cc = 0; cc < w; ++cc) {
            const T v = src[cc];
            Wb[(size_t)cc * ldw + r] = v;
            const kbits_t k = key_of(v);
            if (better(k, rn + cc, bkey, blin)) { bkey = k; blin = rn + cc; }
        }
    }
    for (int cc = tid; cc < w; cc += PT) colused[cc] = 0;
    __syncthreads();

    const int kmax = min(min(m, n), a.chimax);
    const double S = a.rel ? __longlong_as_double((long long)*a.smax) : 0.0;
    const double tau = a.rel ? a.tol * S : a.tol;
    const kbits_t tkey = threadIdx.x == 0 ? tau_key(tau, T()) : 0;  // thread 0 takes the decision

    int p = 0;
    double eps = 0.0;
    for (;;) {
        const int par = p & 1;
        // (1) CTA best: warp reductions, then warp 0 reduces the warp bests and broadcasts the
        //     CTA's candidate into slot [par][g] of every CTA of the cluster.
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const kbits_t ok = __shfl_xor_sync(0xffffffffu, bkey, off);
            const int ol = __shfl_xor_sync(0xffffffffu, blin, off);
            if (better(ok, ol, bkey, blin)) { bkey = ok; blin = ol; }
        }
        if (lane == 0) { wbest[warp].key = bkey; wbest[warp].lin = blin; }
        __syncthreads();
        if (warp == 0) {
            kbits_t k = lane < NWARP ? wbest[lane].key : 0ull;
            int l = lane < NWARP ? wbest[lane].lin : INT_MAX;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const kbits_t ok = __shfl_xor_sync(0xffffffffu, k, off);
                const int ol = __shfl_xor_sync(0xffffffffu, l, off);
                if (better(ok, ol, k, l)) { k = ok; l = ol; }
            }
            Cand<T> mine;
            mine.key = k;
            mine.lin = l;
            mine.pad = 0;
            mine.val = (l != INT_MAX) ? Wb[(size_t)(l % n - c0) * ldw + l / n] : s_zero(T());
            for (int t = lane; t < C; t += 32) *cl.map_shared_rank(cand + par * C + g, t) = mine;
        }
        cl.sync();
        // (2) winner among the C candidates (warp 0), broadcast through wbest[NWARP]
        if (warp == 0) {
            kbits_t k = 0;
            int l = INT_MAX, src = 0;
            for (int t = lane; t < C; t += 32) {
                const Cand<T>& c = cand[par * C + t];
                if (better(c.key, c.lin, k, l)) { k = c.key; l = c.lin; src = t; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const kbits_t ok = __shfl_xor_sync(0xffffffffu, k, off);
                const int ol = __shfl_xor_sync(0xffffffffu, l, off);
                const int os = __shfl_xor_sync(0xffffffffu, src, off);
                if (better(ok, ol, k, l)) { k = ok; l = ol; src = os; }
            }
            if (lane == 0) {
                const T pv = cand[par * C + src].val;
                wbest[NWARP].key = k;
                wbest[NWARP].lin = l;
                wbest[NWARP].pad = src;
                wbest[NWARP].val = pv;
                decide(dec, k, l, pv, p, kmax, tkey);
            }
        }
        __syncthreads();
        const int wlin = wbest[NWARP].lin;
        const int gw = wbest[NWARP].pad;
        const T piv = wbest[NWARP].val;
        if (dec->code) {  // stop: no unused entry left, tolerance or rank cap reached, or non-finite
            if (dec->code == 2 && g == 0 && tid == 0) atomicOr(a.err, DEVERR_NUMERIC);
            eps = dec->eps;
            break;
        }
        const int ri = wlin / n, cj = wlin % n;
        const bool zpiv = dec->zpiv;
        const T inv = dec->inv;
        if (g == 0 && tid == 0) {
            a.piv_rows[p] = ri;
            a.piv_cols[p] = cj;
            a.D[p] = piv;
        }
        // (3) multipliers from the winning column, read from its owner (never written again)
        {
            const T* colp;
            if (SMEMW) {
                const int c0w = (int)(((long long)n * gw) / C);
                colp = cl.map_shared_rank(Wsm, gw) + (size_t)(cj - c0w) * m;
            } else {
                colp = a.W + (size_t)cj * mmax;
            }
            for (int r = tid; r < m; r += PT) {
                T v;
                if (SMEMW) v = colp[r];
                else v = ldcg_val(colp + r);
                lcol[r] = (rowused[r] || r == ri || zpiv) ? s_zero(T()) : s_mul(v, inv);
            }
        }
        for (int cc = tid; cc < w; cc += PT) {
            const T v = Wb[(size_t)cc * ldw + ri];
            prow[cc] = v;
            if (a.U) {
                const int c = c0 + cc;
                T u;
                if (c == cj) u = s_one(T());
                else if (colused[cc] || zpiv) u = s_zero(T());
                else u = s_mul(v, inv);
                a.U[(size_t)p * a.Uld + c] = u;
            }
        }
        __syncthreads();
        if (tid == 0) {
            rowused[ri] = 1;
            if (cj >= c0 && cj < c1) colused[cj - c0] = 1;
        }
        if (a.L) {  // column p of L, rows split across the CTAs
            const int r0 = (int)(((long long)m * g) / C), r1 = (int)(((long long)m * (g + 1)) / C);
            for (int r = r0 + tid; r < r1; r += PT) a.L[(size_t)p * a.Lld + r] = (r == ri) ? s_one(T()) : lcol[r];
        }
        __syncthreads();
        // (4) Schur-complement update (thread = row), fused with the next local argmax
        bkey = 0;
        blin = INT_MAX;
        for (int r = tid; r < m; r += PT) {
            if (rowused[r]) continue;
            const T l = lcol[r];
            const int rn = r * n + c0;
            T* rowp = Wb + r;
            for (int cc = 0; cc < w; ++cc) {
                if (colused[cc]) continue;
                T* ptr = rowp + (size_t)cc * ldw;
                const T v = s_fms(l, prow[cc], *ptr);
                *ptr = v;
                const kbits_t k = key_of(v);
                if (better(k, rn + cc, bkey, blin)) { bkey = k; blin = rn + cc; }
            }
        }
        ++p;
    }
    grid_dependents_launch();  // the next kernel of the stream (a gather) may start launching
    if (g == 0 && tid == 0) {
        if (a.flops) {
            const double per = (sizeof(T) == sizeof(cplx)) ? 8.0 : 2.0;
            const double f = schur_mults(m, n, p);
            atomicAdd(a.flops, per * f);
        }
        *a.eps_out = eps;
        if (a.k_out) *a.k_out = p;
        if (a.out_chi_idx >= 0) const_cast<int*>(a.chi)[a.out_chi_idx] = p;
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------- register-resident cluster variant
// The usual case (cluster sizes up to 16, m <= 1024 rows, at most 32 columns per CTA): each of
// the 512 threads keeps its rows' slice of the CTA's columns in registers, so the Schur update
// is a run of independent FP64 multiply-adds with no shared-memory traffic. Per step:
//   warp maxima -> shared -> every warp reduces them (no broadcast barrier);
//   the CTA writes its candidate column to shared memory and its candidate (key, position,
//   value) into every CTA's slot; one cluster barrier; every warp reduces the C candidates;
//   each thread reads its rows' entries of the winning column from the owner's shared memory;
//   the thread holding the pivot row publishes it; one block barrier; update.
constexpr int RT = 512;
constexpr int RWARP = RT / 32;

__device__ __forceinline__ double shfl_from(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ cplx shfl_from(cplx v, int src) {
    return mkc(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}

// Warp argmax of (key, lowest position) with single-instruction warp reductions: the max of the
// high 32 key bits, then of the low 32 bits among those lanes, then the min position among the
// lanes holding that key; the winner's value and tag travel by one shuffle. The result is the
// same as a pairwise reduction with better(), in three reduction latencies instead of five
// rounds of dependent shuffles.
template <class T>
__device__ __forceinline__ void warp_best(kbits_t& k, int& l, T& v, int& s) {
    const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    const bool top = hi == mhi && lo == mlo;
    const unsigned ml = __reduce_min_sync(0xffffffffu, top ? (unsigned)l : 0xFFFFFFFFu);
    const int src = __ffs(__ballot_sync(0xffffffffu, top && (unsigned)l == ml)) - 1;
    k = ((kbits_t)mhi << 32) | mlo;
    l = (int)ml;
    v = shfl_from(v, src);
    s = __shfl_sync(0xffffffffu, s, src);
}

// Positions of the register-resident kernel: (row << 16) | column. For column < n <= 65536 they
// order like row * n + column, so the lowest-position tie-break is unchanged, and they decode
// with shifts instead of integer divisions on the step's critical path.
__device__ __forceinline__ int cpos(int r, int c) { return (r << 16) + c; }
__device__ __forceinline__ int cpos_row(int p) { return p >> 16; }
__device__ __forceinline__ int cpos_col(int p) { return p & 0xFFFF; }

// v[j] for a runtime j in [0, W) by a tree of selects (log2 W levels instead of a chain of W).
template <class T, int W>
__device__ __forceinline__ T select_reg(const T (&v)[W], int j) {
    T t[W];
#pragma unroll
    for (int c = 0; c < W; ++c) t[c] = v[c];
#pragma unroll
    for (int s = 1; s < W; s <<= 1)
#pragma unroll
        for (int c = 0; c + s < W; c += 2 * s) t[c] = (j & s) ? t[c + s] : t[c];
    return t[0];
}

template <class T, int ROWS, int WMAX>
__global__ void __launch_bounds__(RT, 1) prrlu_creg_kernel(PrrluArgs<T> a) {
    grid_dependency_wait();  // launched early behind the previous kernel of the stream: its outputs are read below
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int g = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = dimv(a.m, a.chi), n = dimv(a.n, a.chi);
    if (small_block(a, m, n)) return;  // every CTA of the cluster returns before any exchange
    const int c0 = (int)(((long long)n * g) / C), c1 = (int)(((long long)n * (g + 1)) / C);
    const int w = c1 - c0;  // <= WMAX (the host sizes WMAX for the capacity)
    const int mmax = a.mmax;

    // shared memory: candcol[2][mmax] | prow[WMAX] | cand[2][C] | warp maxima
    T* candcol = reinterpret_cast<T*>(smem_raw);
    T* prow = candcol + 2 * (size_t)mmax;
    Cand<T>* cand = align16<Cand<T>>(prow + WMAX);
    Cand<T>* wmx = cand + 2 * C;  // [RWARP]
    Decision<T>* dec = reinterpret_cast<Decision<T>*>(wmx + RWARP);

    T v[ROWS][WMAX];
    bool live[ROWS];
    kbits_t bkey = 0;
    int blin = INT_MAX;
    T bval = s_zero(T());
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
        const int r = tid + i * RT;
        live[i] = r < m;
        const T* src = a.Min + (size_t)r * n + c0;
#pragma unroll
        for (int cc = 0; cc < WMAX; ++cc) {
            T x = s_zero(T());
            if (live[i] && cc < w) {
                x = src[cc];
                const kbits_t k = key_of(x);
                const int pos = cpos(r, c0 + cc);
                if (better(k, pos, bkey, blin)) { bkey = k; blin = pos; bval = x; }
            }
            v[i][cc] = x;
        }
    }
    unsigned int colmask = (w >= 32) ? 0xFFFFFFFFu : ((1u << w) - 1u);

    const int kmax = min(min(m, n), a.chimax);
    const double S = a.rel ? __longlong_as_double((long long)*a.smax) : 0.0;
    const double tau = a.rel ? a.tol * S : a.tol;
    const kbits_t tkey = tau_key_cta<T>(tau);  // every warp takes the decision

    int p = 0;
    double eps = 0.0;
    for (;;) {
        const int par = p & 1;
        // (1) the CTA's candidate
        int dummy = 0;
        warp_best(bkey, blin, bval, dummy);
        if (lane == 0) {
            wmx[warp].key = bkey;
            wmx[warp].lin = blin;
            wmx[warp].val = bval;
        }
        __syncthreads();
        kbits_t ck = 0;
        int cl_ = INT_MAX, cs = 0;
        T cv = s_zero(T());
        if (lane < RWARP) { ck = wmx[lane].key; cl_ = wmx[lane].lin; cv = wmx[lane].val; }
        warp_best(ck, cl_, cv, cs);
        const int ccb = (cl_ != INT_MAX) ? (cpos_col(cl_) - c0) : 0;
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            const int r = tid + i * RT;
            if (r < m) candcol[(size_t)par * mmax + r] = select_reg<T, WMAX>(v[i], ccb);
        }
        if (warp == 0) {
            Cand<T> mine;
            mine.key = ck;
            mine.lin = cl_;
            mine.pad = 0;
            mine.val = cv;
            for (int t = lane; t < C; t += 32) *cl.map_shared_rank(cand + par * C + g, t) = mine;
        }
        cl.sync();
        // (2) the winner among the C candidates (C <= 32) and the step's decision, taken by every
        //     warp alike from its own copy of the candidates (integer work, no broadcast barrier)
        kbits_t wk = 0;
        int wl = INT_MAX, gw = 0;
        T pv = s_zero(T());
        if (lane < C) {
            const Cand<T>& c = cand[par * C + lane];
            wk = c.key;
            wl = c.lin;
            pv = c.val;
            gw = lane;
        }
        warp_best(wk, wl, pv, gw);
        Decision<T> dl;
        decide(&dl, wk, wl, pv, p, kmax, tkey, false);
        if (dl.code) {
            if (dl.code == 2 && g == 0 && tid == 0) atomicOr(a.err, DEVERR_NUMERIC);
            eps = dl.eps;
            break;
        }
        const int zpiv = dl.zpiv;
        const int ri = cpos_row(wl), cj = cpos_col(wl);
        if (g == 0 && tid == 0) {
            a.piv_rows[p] = ri;
            a.piv_cols[p] = cj;
            a.D[p] = pv;
        }
        // (3) reads of the winning column from its owner's shared memory start here; thread 0
        //     forms the pivot reciprocal while they are in flight, and it is read after the
        //     barrier that also publishes the pivot row.
        const T* wcol = cl.map_shared_rank(candcol + (size_t)par * mmax, gw);
        T wv[ROWS];
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            const int r = tid + i * RT;
            wv[i] = (live[i] && r != ri && !zpiv) ? wcol[r] : s_zero(T());
            if (r == ri) {  // this thread holds the pivot row: publish it
#pragma unroll
                for (int cc = 0; cc < WMAX; ++cc) prow[cc] = v[i][cc];
                live[i] = false;
            }
        }
        if (tid == 0 && !zpiv) dec->inv = recip_of(pv);
        const unsigned oldmask = colmask;
        if (cj >= c0 && cj < c1) colmask &= ~(1u << (cj - c0));
        __syncthreads();
        const T inv = zpiv ? s_zero(T()) : dec->inv;
        T l[ROWS];
        const int r0 = (int)(((long long)m * g) / C), r1 = (int)(((long long)m * (g + 1)) / C);
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            const int r = tid + i * RT;
            l[i] = s_zero(T());
            if (live[i]) l[i] = s_mul(wv[i], inv);  // no FP64 issue for warps whose rows are all used
            if (a.L && r >= r0 && r < r1) a.L[(size_t)p * a.Lld + r] = (r == ri) ? s_one(T()) : l[i];
        }
        if (a.U && tid < w) {  // row p of U for the own columns, one thread per column
            const int c = c0 + tid;
            T u;
            if (c == cj) u = s_one(T());
            else if (!((oldmask >> tid) & 1u) || zpiv) u = s_zero(T());
            else u = s_mul(prow[tid], inv);
            a.U[(size_t)p * a.Uld + c] = u;
        }
        // (4) Schur-complement update in registers, fused with the next local argmax
        kbits_t qk[4] = {0, 0, 0, 0};
        int ql[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
        T qv[4] = {s_zero(T()), s_zero(T()), s_zero(T()), s_zero(T())};
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            if (!live[i]) continue;
            const int rn = cpos(tid + i * RT, c0);
#pragma unroll
            for (int cc = 0; cc < WMAX; ++cc) {
                if ((colmask >> cc) & 1u) {
                    const T x = s_fms(l[i], prow[cc], v[i][cc]);
                    v[i][cc] = x;
                    const kbits_t k = key_of(x);
                    if (better(k, rn + cc, qk[cc & 3], ql[cc & 3])) { qk[cc & 3] = k; ql[cc & 3] = rn + cc; qv[cc & 3] = x; }
                }
            }
        }
        bkey = qk[0];
        blin = ql[0];
        bval = qv[0];
#pragma unroll
        for (int q = 1; q < 4; ++q)
            if (better(qk[q], ql[q], bkey, blin)) { bkey = qk[q]; blin = ql[q]; bval = qv[q]; }
        ++p;
    }
    grid_dependents_launch();  // the next kernel of the stream (a gather) may start launching
    if (g == 0 && tid == 0) {
        if (a.flops) {
            const double per = (sizeof(T) == sizeof(cplx)) ? 8.0 : 2.0;
            const double f = schur_mults(m, n, p);
            atomicAdd(a.flops, per * f);
        }
        *a.eps_out = eps;
        if (a.k_out) *a.k_out = p;
        if (a.out_chi_idx >= 0) const_cast<int*>(a.chi)[a.out_chi_idx] = p;
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------- 2D register-resident cluster variant
// The C = Cr x Cc CTAs of the cluster tile the block as a Cr x Cc grid: CTA (rg, cg) holds rows
// [R0, R1) and columns [C0, C1) in registers, lane l the rows R0 + l + 32 i, warp w the columns
// C0 + w CC + j. Every CTA sends its candidate into every CTA's slot with st.async stores that
// complete on the receiver's candidate mbarrier of the step's parity (or, with ACI_PRRLU_MBX=0,
// with plain DSMEM stores and the cluster barrier). After the decision only the CTAs holding the
// pivot column send its entries, each to the Cc CTAs of its row group, and only those holding the
// pivot row send theirs, each to the Cr CTAs of its column group, again as st.async stores on the
// receiver's mbarrier: no SM sends more than Cc (R1 - R0) + Cr (C1 - C0) values per step, where the
// 1D split has every CTA read the whole pivot column out of one SM (C m values). Thread 0 forms
// the pivot reciprocal while the values are in flight and arrives on the mbarrier with the
// expected byte count. The multipliers l = S[r, j] / pivot of the CTA's rows and its entries of
// U's row are formed once (one thread per row or column, not once per warp: a warp-wide FP64
// multiply holds an SM sub-partition's FP64 unit ~64 cycles) and shared through one block
// barrier. Every wait is bounded; a run-out wait is reported with the next candidate and every
// CTA stops there. The arithmetic of every entry is that of the other variants, so all of them
// choose the same pivots (bit for bit). Measured against the 1D register variant it is faster on
// complex blocks, on blocks of more than 512 rows and on narrow ones, slower on large square real
// blocks (480 x 480: 1.56 vs 1.36 ms per call), where the FP64 update dominates both.
constexpr int DT = 512;
constexpr int DWARP = DT / 32;

__device__ __forceinline__ uint32_t smem_u32addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// The shared::cluster address of the same offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_async_val(uint32_t addr, double v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr),
                 "l"(__double_as_longlong(v)), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async_val(uint32_t addr, cplx v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b64 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "l"(__double_as_longlong(v.re)), "l"(__double_as_longlong(v.im)), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
constexpr unsigned long long kC2dWaitNs = 1000000000ull;  // 1 s per wait

// A candidate (32 bytes: key, position, flag, value) as two 16-byte st.async stores.
template <class T>
__device__ __forceinline__ void st_async_cand(uint32_t addr, const Cand<T>& c, uint32_t bar) {
    const unsigned long long w1 = ((unsigned long long)(unsigned int)c.pad << 32) | (unsigned int)c.lin;
    unsigned long long w2, w3;
    if constexpr (sizeof(T) == sizeof(double)) {
        w2 = (unsigned long long)__double_as_longlong(reinterpret_cast<const double&>(c.val));
        w3 = 0;
    } else {
        w2 = (unsigned long long)__double_as_longlong(reinterpret_cast<const double*>(&c.val)[0]);
        w3 = (unsigned long long)__double_as_longlong(reinterpret_cast<const double*>(&c.val)[1]);
    }
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b64 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "l"(c.key), "l"(w1), "r"(bar)
                 : "memory");
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b64 [%0], {%1, %2}, [%3];" ::"r"(addr + 16),
                 "l"(w2), "l"(w3), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mb_init(uint32_t bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// Has the phase of parity `parity` completed? Acquire at cluster scope: the st.async values that
// other CTAs sent are visible once it has.
__device__ __forceinline__ bool mb_done_cluster(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, "
        "p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// The same test without the hardware's bounded suspend of try_wait (returns at once).
__device__ __forceinline__ bool mb_test_cluster(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, "
        "p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait (bounded) for the phase of parity `parity`: `polls` > 0 non-blocking tests at most (a
// diagnostic limit, so that a short limit really runs out), else kC2dWaitNs of polling. False
// when the wait ran out.
__device__ __forceinline__ bool mb_wait_bounded(uint32_t bar, uint32_t parity, long long polls) {
    if (polls > 0) {
        for (long long it = 0; it < polls; ++it)
            if (mb_test_cluster(bar, parity)) return true;
        return false;
    }
    if (mb_done_cluster(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned it = 1;; ++it) {
        if (mb_done_cluster(bar, parity)) return true;
        if ((it & 63u) == 0 && globaltimer_ns() - t0 > kC2dWaitNs) return false;
    }
}

// Shared-memory bytes of the 2D variant (rcol, lsm [32 RR] | rrow [DWARP CC] | cand [2][C] |
// warp maxima [DWARP] | 1 / pivot | mbarrier, flags | candidate mbarriers [2] | used rows [32 RR] |
// used columns [DWARP CC]).
template <class T>
__host__ __device__ constexpr size_t c2d_vals_bytes(int rr, int cc) {
    return (sizeof(T) * (2 * 32 * (size_t)rr + (size_t)DWARP * cc) + 15) & ~(size_t)15;
}
template <class T>
size_t c2d_bytes(int rr, int cc, int C) {
    size_t b = c2d_vals_bytes<T>(rr, cc);
    b += sizeof(Cand<T>) * (2 * (size_t)C + DWARP);
    b += ((sizeof(T) + 15) & ~(size_t)15) + 32;
    b += 32 * (size_t)rr + (size_t)DWARP * cc;
    return (b + 15) & ~(size_t)15;
}

template <class T, int RR, int CC>
__global__ void __launch_bounds__(DT, 1) prrlu_c2d_kernel(PrrluArgs<T> a) {
    grid_dependency_wait();  // launched early behind the previous kernel of the stream: its outputs are read below
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int g = (int)cl.block_rank();
    const int Cc = a.grid_c, Cr = C / Cc;
    const int rg = g / Cc, cgr = g - rg * Cc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = dimv(a.m, a.chi), n = dimv(a.n, a.chi);
    if (small_block(a, m, n)) return;  // every CTA of the cluster returns before any exchange
    const int R0 = (int)(((long long)m * rg) / Cr), R1 = (int)(((long long)m * (rg + 1)) / Cr);
    const int C0 = (int)(((long long)n * cgr) / Cc), C1 = (int)(((long long)n * (cgr + 1)) / Cc);
    const int nr = R1 - R0, nc = C1 - C0;  // <= 32 RR and <= DWARP CC (the host sizes RR, CC for the capacity)

    T* rcol = reinterpret_cast<T*>(smem_raw);  // received entries of the pivot column, local rows
    T* lsm = rcol + 32 * RR;                    // multipliers of the local rows
    T* rrow = lsm + 32 * RR;                    // received entries of the pivot row, local columns
    Cand<T>* cand = reinterpret_cast<Cand<T>*>(smem_raw + c2d_vals_bytes<T>(RR, CC));
    Cand<T>* wmx = cand + 2 * C;
    T* sinv = reinterpret_cast<T*>(wmx + DWARP);
    unsigned long long* mbar = align16<unsigned long long>(sinv + 1);  // pushed pivot row and column
    int* sfail = reinterpret_cast<int*>(mbar + 1);      // a wait of this CTA ran out (reported)
    int* shard = sfail + 1;                             // ... and its second, long wait too
    unsigned long long* cbar = mbar + 2;                // [2] candidates by step parity (mbx)
    unsigned char* used_r = reinterpret_cast<unsigned char*>(mbar + 4);
    unsigned char* used_c = used_r + 32 * RR;
    const uint32_t bar = smem_u32addr(mbar), cbar_a = smem_u32addr(cbar);
    const uint32_t rcol_a = smem_u32addr(rcol), rrow_a = smem_u32addr(rrow);
    const bool mbx = a.c2d_mbx != 0;
    if (tid == 0) {
        *sfail = 0;
        *shard = 0;
        mb_init(bar, 1);
        mb_init(cbar_a, 1);
        mb_init(cbar_a + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int t = tid; t < 32 * RR; t += DT) {
        used_r[t] = (unsigned char)(t >= nr);
        lsm[t] = s_zero(T());  // rows past the CTA's own keep a zero multiplier
    }
    for (int t = tid; t < DWARP * CC; t += DT) used_c[t] = (unsigned char)(t >= nc);

    const int cw = C0 + warp * CC;  // this warp's first column
    unsigned int colmask = 0;
#pragma unroll
    for (int j = 0; j < CC; ++j)
        if (cw + j < C1) colmask |= 1u << j;
    // Rows that are not (or no longer) live hold zeros, get a zero multiplier, and take positions
    // past every live one (rb), so the branch-free update leaves them at zero and they can only
    // win the argmax when no live entry is left, which the stop test excludes (p < min(m, n)).
    T v[RR][CC];
    bool live[RR];
    int rb[RR];  // position of the row's entry in column cw (+ j for column cw + j)
    kbits_t bkey = 0;
    int blin = INT_MAX;
    T bval = s_zero(T());
#pragma unroll
    for (int i = 0; i < RR; ++i) {
        const int r = R0 + lane + 32 * i;
        live[i] = r < R1;
        rb[i] = live[i] ? cpos(r, cw) : INT_MAX - CC;
#pragma unroll
        for (int j = 0; j < CC; ++j) {
            T x = s_zero(T());
            if (live[i] && ((colmask >> j) & 1u)) {
                x = a.Min[(size_t)r * n + cw + j];
                const kbits_t k = key_of(x);
                const int pos = cpos(r, cw + j);
                if (better(k, pos, bkey, blin)) { bkey = k; blin = pos; bval = x; }
            }
            v[i][j] = x;
        }
    }

    const int kmax = min(min(m, n), a.chimax);
    const double S = a.rel ? __longlong_as_double((long long)*a.smax) : 0.0;
    const double tau = a.rel ? a.tol * S : a.tol;
    const kbits_t tkey = tau_key_cta<T>(tau);  // every warp takes the decision
    const uint32_t rbytes = (uint32_t)(((size_t)nr + (size_t)nc) * sizeof(T));
    if (mbx) cl.sync();  // every CTA's mbarriers are initialised before any CTA signals one

    int p = 0;
    double eps = 0.0;
    for (;;) {
        const int par = p & 1;
        const uint32_t cb = cbar_a + 8u * (uint32_t)par;
        if (mbx && tid == 0) mb_arrive_expect(cb, (uint32_t)(C * sizeof(Cand<T>)));
        // (1) the CTA's candidate, and its copy into every CTA's slots
        int dummy = 0;
        warp_best(bkey, blin, bval, dummy);
        if (lane == 0) {
            wmx[warp].key = bkey;
            wmx[warp].lin = blin;
            wmx[warp].val = bval;
        }
        __syncthreads();
        if (warp == 0) {
            kbits_t ck = 0;
            int cl_ = INT_MAX, cs = 0;
            T cv = s_zero(T());
            if (lane < DWARP) { ck = wmx[lane].key; cl_ = wmx[lane].lin; cv = wmx[lane].val; }
            warp_best(ck, cl_, cv, cs);
            Cand<T> mine;
            mine.key = ck;
            mine.lin = cl_;
            mine.pad = *sfail;
            mine.val = cv;
            if (mbx) {
                const uint32_t slot = smem_u32addr(cand + par * C + g);
                for (int t = lane; t < C; t += 32) st_async_cand(peer_addr(slot, t), mine, peer_addr(cb, t));
            } else {
                for (int t = lane; t < C; t += 32) *cl.map_shared_rank(cand + par * C + g, t) = mine;
            }
        }
        if (mbx) {
            // warp 0 waits for the C candidates; the block barrier passes its view (and the outcome,
            // so that every thread of the CTA takes the same branch) to the other warps
            if (warp == 0) {
                const uint32_t cpar = (uint32_t)((p >> 1) & 1);
                bool ok = mb_wait_bounded(cb, cpar, a.spin_limit);
                if (!ok) {
                    if (lane == 0) *sfail = 1;
                    ok = mb_wait_bounded(cb, cpar, 0);
                }
                if (!__all_sync(0xffffffffu, ok) && lane == 0) *shard = 1;
            }
            __syncthreads();
            if (*shard) {  // the exchange itself failed: this CTA stops, the others' waits run out
                if (g == 0 && tid == 0) atomicOr(a.err, DEVERR_TIMEOUT);
                break;
            }
        } else {
            cl.sync();
        }
        // (2) the winner among the C candidates and the step's decision, taken by every warp alike
        kbits_t wk = 0;
        int wl = INT_MAX, gw = 0, bad = 0;
        T pv = s_zero(T());
        if (lane < C) {
            const Cand<T>& c = cand[par * C + lane];
            wk = c.key;
            wl = c.lin;
            pv = c.val;
            gw = lane;
            bad = c.pad;
        }
        if (__any_sync(0xffffffffu, bad)) {  // a CTA's previous wait ran out: every CTA stops here
            if (g == 0 && tid == 0) atomicOr(a.err, DEVERR_TIMEOUT);
            break;
        }
        warp_best(wk, wl, pv, gw);
        Decision<T> dl;
        decide(&dl, wk, wl, pv, p, kmax, tkey, false);
        if (dl.code) {
            if (dl.code == 2 && g == 0 && tid == 0) atomicOr(a.err, DEVERR_NUMERIC);
            eps = dl.eps;
            break;
        }
        const int zpiv = dl.zpiv;
        const int ri = cpos_row(wl), cj = cpos_col(wl);
        if (g == 0 && tid == 0) {
            a.piv_rows[p] = ri;
            a.piv_cols[p] = cj;
            a.D[p] = pv;
        }
        // (3) the pivot column's entries of rows [R0, R1) to the Cc CTAs of this row group (sent by
        //     the warp holding the column), the pivot row's entries of columns [C0, C1) to the Cr
        //     CTAs of this column group (every warp sends its CC of them)
        if (cj >= C0 && cj < C1 && warp == (cj - C0) / CC) {
            const int jc = cj - cw;
#pragma unroll
            for (int i = 0; i < RR; ++i) {
                const int rl = lane + 32 * i;
                if (rl < nr) {
                    const T x = select_reg<T, CC>(v[i], jc);
                    const uint32_t la = rcol_a + (uint32_t)(rl * sizeof(T));
                    for (int q = 0; q < Cc; ++q) {
                        const int dst = rg * Cc + q;
                        st_async_val(peer_addr(la, dst), x, peer_addr(bar, dst));
                    }
                }
            }
        }
        if (ri >= R0 && ri < R1) {
            const int rl = ri - R0, li = rl & 31, ii = rl >> 5;
            T rv[CC];
#pragma unroll
            for (int j = 0; j < CC; ++j) {
                T x = v[0][j];
#pragma unroll
                for (int i = 1; i < RR; ++i)
                    if (i == ii) x = v[i][j];
                rv[j] = shfl_from(x, li);
            }
            for (int q = lane; q < CC * Cr; q += 32) {
                const int j = q % CC, d = q / CC;
                const int cloc = warp * CC + j;  // local column
                if (cloc < nc) {
                    const T x = select_reg<T, CC>(rv, j);
                    const int dst = d * Cc + cgr;
                    st_async_val(peer_addr(rrow_a + (uint32_t)(cloc * sizeof(T)), dst), x, peer_addr(bar, dst));
                }
            }
        }
        // (4) thread 0 forms 1 / pivot while the entries are in flight, then arrives with the byte
        //     count this CTA receives. Only the warps that form multipliers or U entries from the
        //     received entries wait for the phase (bounded); the block barrier below orders what
        //     they saw before the other warps' reads.
        if (tid == 0) {
            *sinv = zpiv ? s_zero(T()) : recip_of(pv);
            mb_arrive_expect(bar, rbytes);
        }
        const int uw0 = (DT - DWARP * CC) >> 5;  // first warp of the U entries
        const bool lrole = warp < ((nr + 31) >> 5);
        const bool urole = warp >= uw0 && warp < uw0 + ((nc + 31) >> 5);
        if (lrole || urole) {
            // a run-out wait is reported with the next candidate (every CTA then stops there) and
            // waited out again with the long bound, so that no entry is still in flight to this CTA
            bool ok = mb_wait_bounded(bar, (uint32_t)par, a.spin_limit);
            if (!ok) {
                *sfail = 1;
                ok = mb_wait_bounded(bar, (uint32_t)par, 0);
            }
            if (!ok) *shard = 1;
        }
        const T inv = *sinv;
        // (5) multipliers of the local rows and this CTA's entries of row p of U, one thread each
        if (tid < nr) {
            const int r = R0 + tid;
            T l = s_zero(T());
            if (r == ri) used_r[tid] = 1;
            else if (!used_r[tid]) l = s_mul(rcol[tid], inv);
            lsm[tid] = l;
            if (a.L && cgr == 0) a.L[(size_t)p * a.Lld + r] = (r == ri) ? s_one(T()) : l;
        }
        if (tid >= DT - DWARP * CC && tid - (DT - DWARP * CC) < nc) {
            const int t = tid - (DT - DWARP * CC), c = C0 + t;
            T u = s_zero(T());
            if (c == cj) {
                u = s_one(T());
                used_c[t] = 1;
            } else if (!used_c[t] && !zpiv) {
                u = s_mul(rrow[t], inv);
            }
            if (a.U && rg == 0) a.U[(size_t)p * a.Uld + c] = u;
        }
#pragma unroll
        for (int i = 0; i < RR; ++i)
            if (R0 + lane + 32 * i == ri) {
                live[i] = false;
                rb[i] = INT_MAX - CC;
#pragma unroll
                for (int j = 0; j < CC; ++j) v[i][j] = s_zero(T());
            }
        if (cj >= cw && cj < cw + CC) colmask &= ~(1u << (cj - cw));
        __syncthreads();
        if (mbx && *shard) {  // (with the cluster barrier the steps stay in lockstep instead)
            if (g == 0 && tid == 0) atomicOr(a.err, DEVERR_TIMEOUT);
            break;
        }
        // (6) Schur-complement update in registers, fused with the next local argmax: one chain per
        //     row slot; along a row the positions grow with j, so a later entry wins only with a
        //     strictly larger key, and the chain keeps the key and the column index alone. The
        //     first live column is the chain's start, which makes a row of zeros report its lowest
        //     live position.
        T u[CC];
#pragma unroll
        for (int j = 0; j < CC; ++j) u[j] = rrow[warp * CC + j];
        const int jfirst = __ffs(colmask) - 1;
        kbits_t qk[RR];
        int qj[RR];
#pragma unroll
        for (int i = 0; i < RR; ++i) {
            qk[i] = 0;
            qj[i] = jfirst;
            if (!__any_sync(0xffffffffu, live[i])) continue;  // warp-uniform: no live row in this slot
            const T li = lsm[lane + 32 * i];
#pragma unroll
            for (int j = 0; j < CC; ++j) {
                if ((colmask >> j) & 1u) {
                    const T x = s_fms(li, u[j], v[i][j]);
                    v[i][j] = x;
                    const kbits_t k = key_of(x);
                    if (k > qk[i]) { qk[i] = k; qj[i] = j; }
                }
            }
        }
        bkey = 0;
        blin = INT_MAX;
        bval = s_zero(T());
        if (colmask) {
#pragma unroll
            for (int i = 0; i < RR; ++i) {
                const int pos = rb[i] + qj[i];
                if (better(qk[i], pos, bkey, blin)) {
                    bkey = qk[i];
                    blin = pos;
                    bval = select_reg<T, CC>(v[i], qj[i]);
                }
            }
        }
        ++p;
    }
    grid_dependents_launch();  // the next kernel of the stream (a gather) may start launching
    if (g == 0 && tid == 0) {
        if (a.flops) {
            const double per = (sizeof(T) == sizeof(cplx)) ? 8.0 : 2.0;
            const double f = schur_mults(m, n, p);
            atomicAdd(a.flops, per * f);
        }
        *a.eps_out = eps;
        if (a.k_out) *a.k_out = p;
        if (a.out_chi_idx >= 0) const_cast<int*>(a.chi)[a.out_chi_idx] = p;
    }
    cl.sync();  // no CTA leaves while another may still write into its shared memory
}

// ---------------------------------------------------------------- single-CTA variant
// Small live blocks (most bonds of a chain whose ranks fall away from the middle, whatever the
// capacity the launch was sized for): the whole block in the registers of one CTA of CT threads,
// so a pivot step needs neither a cluster barrier nor distributed shared memory. Warp w holds the
// column chunk [w W, w W + W) of every row, lane l the rows l, l + 32, ..., l + 32 (ROWS - 1).
// Per step: the warp argmax of the per-thread bests (fused in the update) -> shared memory -> one
// block barrier -> every warp reduces the warp maxima and takes the step's decision itself; the
// warp holding the pivot column and the lanes holding the pivot row publish them -> a second block
// barrier -> multipliers, L and U entries and the register update. The arithmetic of every entry
// is that of the other variants (l = S[r, j] x (1 / pivot), S[r, c] - l S[i, c] fused), so the
// variants choose the same pivots.
constexpr int CT = 256;
constexpr int CWARP = CT / 32;

template <class T, int ROWS, int W>
__global__ void __launch_bounds__(CT, 1) prrlu_cta_kernel(PrrluArgs<T> a) {
    grid_dependency_wait();  // launched early behind the previous kernel of the stream: its outputs are read below
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = dimv(a.m, a.chi), n = dimv(a.n, a.chi);
    if (!small_block(a, m, n)) return;  // the capacity's variant takes this block

    // shared memory: lcol[2][32 ROWS] | prow[2][CWARP W] | 1 / pivot [2] | warp maxima [2][CWARP]
    T* lcol = reinterpret_cast<T*>(smem_raw);
    T* prow = lcol + 2 * 32 * ROWS;
    T* sinv = prow + 2 * CWARP * W;
    Cand<T>* wmx = align16<Cand<T>>(sinv + 2);
    const int c0 = warp * W;

    T v[ROWS][W];
    bool live[ROWS];
    kbits_t bkey = 0;
    int blin = INT_MAX;
    T bval = s_zero(T());
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
        const int r = lane + 32 * i;
        live[i] = r < m;
#pragma unroll
        for (int c = 0; c < W; ++c) {
            T x = s_zero(T());
            if (live[i] && c0 + c < n) {
                x = a.Min[(size_t)r * n + c0 + c];
                const kbits_t k = key_of(x);
                const int pos = cpos(r, c0 + c);
                if (better(k, pos, bkey, blin)) { bkey = k; blin = pos; bval = x; }
            }
            v[i][c] = x;
        }
    }
    unsigned int colmask = 0;
#pragma unroll
    for (int c = 0; c < W; ++c)
        if (c0 + c < n) colmask |= 1u << c;

    const int kmax = min(min(m, n), a.chimax);
    const double S = a.rel ? __longlong_as_double((long long)*a.smax) : 0.0;
    const double tau = a.rel ? a.tol * S : a.tol;
    const kbits_t tkey = tau_key_cta<T>(tau);  // every warp takes the decision

    int p = 0;
    double eps = 0.0;
    for (;;) {
        const int par = p & 1;
        int dummy = 0;
        warp_best(bkey, blin, bval, dummy);
        if (lane == 0) {
            Cand<T> mine;
            mine.key = bkey;
            mine.lin = blin;
            mine.pad = 0;
            mine.val = bval;
            wmx[par * CWARP + warp] = mine;
        }
        __syncthreads();
        // the step's winner and decision, taken by every warp from the warp maxima
        kbits_t wk = 0;
        int wl = INT_MAX, gw = 0;
        T pv = s_zero(T());
        if (lane < CWARP) {
            const Cand<T> c = wmx[par * CWARP + lane];
            wk = c.key;
            wl = c.lin;
            pv = c.val;
            gw = lane;
        }
        warp_best(wk, wl, pv, gw);
        Decision<T> dl;
        decide(&dl, wk, wl, pv, p, kmax, tkey, false);
        if (dl.code) {
            if (dl.code == 2 && tid == 0) atomicOr(a.err, DEVERR_NUMERIC);
            eps = dl.eps;
            break;
        }
        const int zpiv = dl.zpiv;
        const int ri = cpos_row(wl), cj = cpos_col(wl);
        if (tid == 0) {
            a.piv_rows[p] = ri;
            a.piv_cols[p] = cj;
            a.D[p] = pv;
        }
        // publish the pivot column (its warp) and the pivot row (its lane in every warp)
        T* lc = lcol + par * 32 * ROWS;
        T* pr = prow + par * CWARP * W;
        if (warp == cj / W) {
#pragma unroll
            for (int i = 0; i < ROWS; ++i) lc[lane + 32 * i] = select_reg<T, W>(v[i], cj - c0);
        }
        if (lane == (ri & 31)) {
            const int i0 = ri >> 5;
#pragma unroll
            for (int c = 0; c < W; ++c) {
                T x = v[0][c];
#pragma unroll
                for (int i = 1; i < ROWS; ++i)
                    if (i == i0) x = v[i][c];
                pr[c0 + c] = x;
            }
        }
#pragma unroll
        for (int i = 0; i < ROWS; ++i)
            if (lane + 32 * i == ri) live[i] = false;
        const unsigned oldmask = colmask;
        if (warp == cj / W) colmask &= ~(1u << (cj - c0));
        // one thread forms the reciprocal (FP64 issue slots are scarce: 2 multiply-adds per clock
        // per SM), the block barrier below publishes it
        if (tid == 0) sinv[par] = zpiv ? s_zero(T()) : recip_of(pv);
        __syncthreads();
        const T inv = sinv[par];
        T l[ROWS];
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            const int r = lane + 32 * i;
            l[i] = s_zero(T());
            if (live[i] && !zpiv) l[i] = s_mul(lc[r], inv);
            if (a.L && warp == 0 && r < m) a.L[(size_t)p * a.Lld + r] = (r == ri) ? s_one(T()) : l[i];
        }
        if (a.U && lane < W && c0 + lane < n) {  // row p of U over this warp's columns
            const int c = c0 + lane;
            T u;
            if (c == cj) u = s_one(T());
            else if (!((oldmask >> lane) & 1u) || zpiv) u = s_zero(T());
            else u = s_mul(pr[c], inv);
            a.U[(size_t)p * a.Uld + c] = u;
        }
        T u[W];
#pragma unroll
        for (int c = 0; c < W; ++c) u[c] = pr[c0 + c];
        // Schur-complement update in registers, fused with the next local argmax (4 chains)
        kbits_t qk[4] = {0, 0, 0, 0};
        int ql[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
        T qv[4] = {s_zero(T()), s_zero(T()), s_zero(T()), s_zero(T())};
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            if (!live[i]) continue;
            const int rn = cpos(lane + 32 * i, c0);
#pragma unroll
            for (int c = 0; c < W; ++c) {
                if ((colmask >> c) & 1u) {
                    const T x = s_fms(l[i], u[c], v[i][c]);
                    v[i][c] = x;
                    const kbits_t k = key_of(x);
                    if (better(k, rn + c, qk[c & 3], ql[c & 3])) { qk[c & 3] = k; ql[c & 3] = rn + c; qv[c & 3] = x; }
                }
            }
        }
        bkey = qk[0];
        blin = ql[0];
        bval = qv[0];
#pragma unroll
        for (int q = 1; q < 4; ++q)
            if (better(qk[q], ql[q], bkey, blin)) { bkey = qk[q]; blin = ql[q]; bval = qv[q]; }
        ++p;
    }
    grid_dependents_launch();  // the next kernel of the stream (a gather) may start launching
    if (tid == 0) {
        if (a.flops) {
            const double per = (sizeof(T) == sizeof(cplx)) ? 8.0 : 2.0;
            const double f = schur_mults(m, n, p);
            atomicAdd(a.flops, per * f);
        }
        *a.eps_out = eps;
        if (a.k_out) *a.k_out = p;
        if (a.out_chi_idx >= 0) const_cast<int*>(a.chi)[a.out_chi_idx] = p;
    }
}

// ---------------------------------------------------------------- rook search (second pivot mode)
//
// The rook variant of Algorithm 2's pivot search. The residual
//   R_p = M - sum_{q<p} L[:, q] D[q] U[q, :]
// is never formed as a whole: each hop evaluates one column (or row) of it, a matrix-vector
// product with the stored factors, and takes its argmax over the unused rows (columns). From the
// start column c0: r1 = argmax_r |R(r,c0)|, c1 = argmax_c |R(r1,c)|; c1 == c0 accepts (r1, c0);
// else r2 = argmax_r |R(r,c1)|; r2 == r1 accepts (r1, c1), otherwise (r2, c1) after a fourth hop
// (the row r2 is evaluated for U). Step 0 starts from the column of the global argmax of |M|,
// step p from the largest residual of the previous pivot row among unused columns. Work per
// step is O((m + n) p) instead of the O(m n) Schur update of the full search.
//
// One persistent cooperative grid. A hop's evaluation splits the rows (columns) into blocks of
// RKB, each handled by one CTA with RKQ partial sums per row (q strided), so L (column-major) and
// U (row-major) are read coalesced; a CTA owns the same rows and columns at every step, writes
// their L and U entries and keeps their used flags, so nothing it reads from L or U was written
// by another CTA except the pivot row of L and the start column of U, which are read after an
// exchange (or, for the newest U row, re-derived from the previous step's residual row). Each
// hop ends in a grid-wide (key, index) argmax: every CTA publishes its best (two best for rows:
// the second gives the next start column) as tagged words and gathers all records (bounded waits).
constexpr int RKT = 256;          // threads per CTA
constexpr int RKB = 16;           // rows (columns) per evaluation block
constexpr int RKQ = RKT / RKB;    // partial sums per row, q = j, j + RKQ, ...
constexpr int RK_REC = 16;        // words per record (one 128-byte line): ready tag, key, index, key2, index2, value
constexpr int RK_AREAS = 5;       // global argmax, column, row, second column, second row

// The two best (key, index) pairs seen, with the best one's value.
template <class T> struct RkCand {
    kbits_t k1;
    int i1;
    kbits_t k2;
    int i2;
    T v1;
};

template <class T>
__device__ __forceinline__ void rk_push(kbits_t k, int i, T v, RkCand<T>& c) {
    if (i == INT_MAX) return;
    if (better(k, i, c.k1, c.i1)) {
        c.k2 = c.k1;
        c.i2 = c.i1;
        c.k1 = k;
        c.i1 = i;
        c.v1 = v;
    } else if (better(k, i, c.k2, c.i2)) {
        c.k2 = k;
        c.i2 = i;
    }
}
template <class T> __device__ __forceinline__ RkCand<T> rk_none() {
    return RkCand<T>{0ull, INT_MAX, 0ull, INT_MAX, s_zero(T())};
}
__device__ __forceinline__ double shfl_val(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ cplx shfl_val(cplx v, int off) {
    return mkc(__shfl_xor_sync(0xffffffffu, v.re, off), __shfl_xor_sync(0xffffffffu, v.im, off));
}
template <class T> __device__ __forceinline__ void rk_warp_merge(RkCand<T>& c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const kbits_t k1 = __shfl_xor_sync(0xffffffffu, c.k1, off);
        const int i1 = __shfl_xor_sync(0xffffffffu, c.i1, off);
        const kbits_t k2 = __shfl_xor_sync(0xffffffffu, c.k2, off);
        const int i2 = __shfl_xor_sync(0xffffffffu, c.i2, off);
        const T v1 = shfl_val(c.v1, off);
        rk_push(k1, i1, v1, c);
        rk_push(k2, i2, s_zero(T()), c);
    }
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void rk_put_val(unsigned long long* p, double v) {
    st_relaxed_u64(p, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void rk_put_val(unsigned long long* p, cplx v) {
    st_relaxed_u64(p, (unsigned long long)__double_as_longlong(v.re));
    st_relaxed_u64(p + 1, (unsigned long long)__double_as_longlong(v.im));
}
__device__ __forceinline__ void rk_get_val(const unsigned long long* p, double& v) { v = __longlong_as_double((long long)ld_word(p)); }
__device__ __forceinline__ void rk_get_val(const unsigned long long* p, cplx& v) {
    v = mkc(__longlong_as_double((long long)ld_word(p)), __longlong_as_double((long long)ld_word(p + 1)));
}

// Publish this CTA's candidates under `tag`, then gather every CTA's record: the grid's two best
// with the best one's value, returned to every thread. A record is one 128-byte line: the data
// words, then a ready word holding the tag, stored with release semantics after a fence that
// orders the CTA's earlier global writes (residual buffers, L, U; the barrier before it collects
// them from every thread). Each thread polls the ready words of its records (relaxed loads, then
// one acquire fence) and reads each record once; the closing barrier passes the acquired view to
// the whole CTA. false: a wait ran out.
template <class T>
__device__ bool rk_exchange(unsigned long long* area, unsigned int tag, RkCand<T> mine, RkCand<T>& out,
                            RkCand<T>* s, int* sok) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    rk_warp_merge(mine);
    if (lane == 0) s[warp] = mine;
    __syncthreads();
    if (warp == 0) {
        RkCand<T> c = lane < RKT / 32 ? s[lane] : rk_none<T>();
        rk_warp_merge(c);
        if (lane == 0) {
            unsigned long long* rec = area + (size_t)blockIdx.x * RK_REC;
            fence_acq_rel_gpu();
            st_relaxed_u64(rec + 1, c.k1);
            st_relaxed_u64(rec + 2, (unsigned long long)(unsigned int)c.i1);
            st_relaxed_u64(rec + 3, c.k2);
            st_relaxed_u64(rec + 4, (unsigned long long)(unsigned int)c.i2);
            rk_put_val(rec + 5, c.v1);
            st_release_u64(rec, tag);
        }
    }
    // every thread gathers records t, t + RKT, ... (one round trip for the ready word, one for the data)
    RkCand<T> g = rk_none<T>();
    bool ok = true;
    for (int t = threadIdx.x; t < (int)gridDim.x && ok; t += RKT) {
        const unsigned long long* rec = area + (size_t)t * RK_REC;
        long long spins = 0;
        while (ld_word(rec) != (unsigned long long)tag) {  // relaxed polling; one acquire fence after
            if (++spins > kSpinLimit) {
                ok = false;
                break;
            }
        }
        if (!ok) break;
        fence_acq_rel_gpu();
        T v;
        rk_get_val(rec + 5, v);
        rk_push(ld_word(rec + 1), (int)(unsigned int)ld_word(rec + 2), v, g);
        rk_push(ld_word(rec + 3), (int)(unsigned int)ld_word(rec + 4), s_zero(T()), g);
    }
    ok = __syncthreads_and(ok);
    rk_warp_merge(g);
    if (lane == 0) s[warp] = g;
    __syncthreads();
    if (warp == 0) {
        g = lane < RKT / 32 ? s[lane] : rk_none<T>();
        rk_warp_merge(g);
        if (lane == 0) {
            s[RKT / 32] = g;
            *sok = ok;
        }
    }
    __syncthreads();
    out = s[RKT / 32];
    return *sok != 0;
}

__device__ __forceinline__ double rk_sub(double a, double b) { return a - b; }
__device__ __forceinline__ cplx rk_sub(cplx a, cplx b) { return mkc(a.re - b.re, a.im - b.im); }

// Residual column c over this CTA's rows: buf[r] = M[r, c] - sum_{q<p} L[r, q] w[q]; the CTA's
// best unused row. (Row evaluation is the same with the roles of the factors exchanged.)
template <class T, bool COL>
__device__ RkCand<T> rk_eval(const PrrluArgs<T>& a, const unsigned char* used, int len, int ldm, int fixed, int p,
                             const T* w, T* part, T* buf) {
    RkCand<T> best = rk_none<T>();
    const int j = threadIdx.x % RKB, qc = threadIdx.x / RKB;
    for (int blk = blockIdx.x; blk * RKB < len; blk += gridDim.x) {
        const int x = blk * RKB + j;  // the row (COL) or column (row evaluation)
        T acc = s_zero(T());
        if (x < len) {
            if (COL) {
#pragma unroll 4
                for (int q = qc; q < p; q += RKQ) acc = s_fma(a.L[(size_t)q * a.Lld + x], w[q], acc);
            } else {
#pragma unroll 4
                for (int q = qc; q < p; q += RKQ) acc = s_fma(w[q], a.U[(size_t)q * a.Uld + x], acc);
            }
        }
        part[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x < RKB && x < len) {
            T sum = part[threadIdx.x];
            for (int t = 1; t < RKQ; ++t) sum = s_add(sum, part[threadIdx.x + t * RKB]);
            const T mv = COL ? a.Min[(size_t)x * ldm + fixed] : a.Min[(size_t)fixed * ldm + x];
            const T R = rk_sub(mv, sum);
            buf[x] = R;
            if (!used[x]) rk_push(key_of(R), x, R, best);
        }
        __syncthreads();
    }
    return best;
}

template <class T>
__global__ void __launch_bounds__(RKT, 1) prrlu_rook_kernel(PrrluArgs<T> a) {
    grid_dependency_wait();  // launched early behind the previous kernel of the stream: its outputs are read below
    extern __shared__ __align__(16) unsigned char rk_smem[];
    const int kcap_s = a.wcap_cols;  // shared capacity of the pivot and weight vectors
    T* Ds = reinterpret_cast<T*>(rk_smem);
    T* w = Ds + kcap_s;
    T* part = w + kcap_s;
    RkCand<T>* sc = align16<RkCand<T>>(part + RKT);
    Decision<T>* dec = align16<Decision<T>>(sc + RKT / 32 + 1);
    int* sok = reinterpret_cast<int*>(dec + 1);
    const int m = dimv(a.m, a.chi), n = dimv(a.n, a.chi);
    const int ldm = n;
    const int kmin = m < n ? m : n;
    const double S = a.rel ? __longlong_as_double((long long)*a.smax) : 0.0;
    const double tau = a.rel ? a.tol * S : a.tol;
    const kbits_t tkey = threadIdx.x == 0 ? tau_key(tau, T()) : 0;  // thread 0 takes the decision
    // scratch: two residual columns, two residual rows, used flags (see prrlu_rook_scratch_bytes)
    T* colbuf[2] = {a.W, a.W + a.mmax};
    T* rowbuf[2] = {a.W + 2 * (size_t)a.mmax, a.W + 2 * (size_t)a.mmax + a.nmax};
    unsigned char* used_r = reinterpret_cast<unsigned char*>(a.W + 2 * (size_t)a.mmax + 2 * (size_t)a.nmax);
    unsigned char* used_c = used_r + a.mmax;
    unsigned long long* area[RK_AREAS];
    for (int i = 0; i < RK_AREAS; ++i) area[i] = a.ll + (size_t)i * gridDim.x * RK_REC;
    const double per = sizeof(T) == sizeof(cplx) ? 8.0 : 2.0;
    double flops = 0.0;

    for (int blk = blockIdx.x; blk * RKB < m; blk += gridDim.x)
        if (threadIdx.x < RKB && blk * RKB + (int)threadIdx.x < m) used_r[blk * RKB + threadIdx.x] = 0;
    for (int blk = blockIdx.x; blk * RKB < n; blk += gridDim.x)
        if (threadIdx.x < RKB && blk * RKB + (int)threadIdx.x < n) used_c[blk * RKB + threadIdx.x] = 0;

    int p = 0, c0 = 0, prev_row = 0;
    T prev_inv = s_zero(T());
    int prev_zero = 0;
    int code = 1;
    double eps = 0.0;
    bool ok = true;
    for (;; ++p) {
        if (p == kmin) {
            code = 1;
            eps = 0.0;
            break;
        }
        const unsigned int tag = a.tagbase + (unsigned int)p + 1;
        RkCand<T> g;
        if (p == 0) {  // start column: the column of the global argmax of |M| (ties: lowest row * n + col)
            RkCand<T> mine = rk_none<T>();
            const long long mn = (long long)m * n;
            for (long long e = (long long)blockIdx.x * RKT + threadIdx.x; e < mn; e += (long long)gridDim.x * RKT)
                rk_push(key_of(a.Min[e]), (int)e, s_zero(T()), mine);
            if (!(ok = rk_exchange(area[0], tag, mine, g, sc, sok))) break;
            c0 = g.i1 == INT_MAX ? 0 : g.i1 % n;
        }
        // weights of the start column: w[q] = D[q] U[q, c0]; the newest U row comes from the previous
        // step's residual row with the arithmetic its writers used
        for (int q = threadIdx.x; q < p; q += RKT) {
            T u;
            if (q < p - 1) {
                u = ldcg_val(a.U + (size_t)q * a.Uld + c0);
            } else {
                u = prev_zero ? s_zero(T()) : s_mul(ldcg_val(rowbuf[prev_row] + c0), prev_inv);
            }
            w[q] = s_mul(Ds[q], u);
        }
        __syncthreads();
        // hop 1: column c0
        RkCand<T> best = rk_eval<T, true>(a, used_r, m, ldm, c0, p, w, part, colbuf[0]);
        flops += per * m * (double)p;
        if (!(ok = rk_exchange(area[1], tag, best, g, sc, sok))) break;
        const int r1 = g.i1;
        T pv = g.v1;  // residual at (r1, c0): the pivot if the search stops here
        // hop 2: row r1
        for (int q = threadIdx.x; q < p; q += RKT) w[q] = s_mul(ldcg_val(a.L + (size_t)q * a.Lld + r1), Ds[q]);
        __syncthreads();
        best = rk_eval<T, false>(a, used_c, n, ldm, r1, p, w, part, rowbuf[0]);
        flops += per * n * (double)p;
        RkCand<T> row1;
        if (!(ok = rk_exchange(area[2], tag, best, row1, sc, sok))) break;
        int r = r1, c = c0, ci = 0, ri = 0;
        RkCand<T> rowsel = row1;
        if (row1.i1 != c0) {
            const int c1 = row1.i1;
            // hop 3: column c1 (every U row it needs has been published by now)
            for (int q = threadIdx.x; q < p; q += RKT)
                w[q] = s_mul(Ds[q], ldcg_val(a.U + (size_t)q * a.Uld + c1));
            __syncthreads();
            best = rk_eval<T, true>(a, used_r, m, ldm, c1, p, w, part, colbuf[1]);
            flops += per * m * (double)p;
            if (!(ok = rk_exchange(area[3], tag, best, g, sc, sok))) break;
            const int r2 = g.i1;
            pv = g.v1;  // the pivot lies in column c1, at r2 (== r1 at a fixed point)
            c = c1;
            ci = 1;
            if (r2 != r1) {
                // hop 4: row r2, for the pivot's U row
                for (int q = threadIdx.x; q < p; q += RKT)
                    w[q] = s_mul(ldcg_val(a.L + (size_t)q * a.Lld + r2), Ds[q]);
                __syncthreads();
                best = rk_eval<T, false>(a, used_c, n, ldm, r2, p, w, part, rowbuf[1]);
                flops += per * n * (double)p;
                if (!(ok = rk_exchange(area[4], tag, best, rowsel, sc, sok))) break;
                r = r2;
                ri = 1;
            }
        }
        // the pivot and the stop test (Algorithm 2, reading R2 with the rook pivot)
        if (threadIdx.x == 0) {
            decide(dec, key_of(pv), r, pv, p, a.chimax, tkey);
            dec->piv = pv;
        }
        __syncthreads();
        if (dec->code != 0) {
            code = dec->code;
            eps = dec->eps;
            break;
        }
        const T piv = dec->piv, inv = dec->inv;
        const int zp = dec->zpiv;
        // L column p over this CTA's rows, U row p over its columns; zero on used rows / columns
        for (int blk = blockIdx.x; blk * RKB < m; blk += gridDim.x) {
            const int x = blk * RKB + (int)threadIdx.x;
            if (threadIdx.x < RKB && x < m) {
                T l;
                if (x == r) l = s_one(T());
                else if (zp || used_r[x]) l = s_zero(T());
                else l = s_mul(colbuf[ci][x], inv);
                a.L[(size_t)p * a.Lld + x] = l;
                if (x == r) used_r[x] = 1;
            }
        }
        for (int blk = blockIdx.x; blk * RKB < n; blk += gridDim.x) {
            const int x = blk * RKB + (int)threadIdx.x;
            if (threadIdx.x < RKB && x < n) {
                T u;
                if (x == c) u = s_one(T());
                else if (zp || used_c[x]) u = s_zero(T());
                else u = s_mul(rowbuf[ri][x], inv);
                a.U[(size_t)p * a.Uld + x] = u;
                if (x == c) used_c[x] = 1;
            }
        }
        if (threadIdx.x == 0) {
            Ds[p] = piv;
            if (blockIdx.x == 0) {
                a.D[p] = piv;
                a.piv_rows[p] = r;
                a.piv_cols[p] = c;
            }
        }
        // next start column: the largest residual of this pivot row among the unused columns
        c0 = rowsel.i1 != c ? rowsel.i1 : rowsel.i2;
        if (c0 == INT_MAX) c0 = 0;  // no unused column left: the next step stops at p == min(m, n)
        prev_row = ri;
        prev_inv = inv;
        prev_zero = zp;
        __syncthreads();
    }
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(a.err, DEVERR_TIMEOUT);
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (code == 2) atomicOr(a.err, DEVERR_NUMERIC);
        *a.eps_out = eps;
        if (a.k_out) *a.k_out = p;
        if (a.out_chi_idx >= 0) const_cast<int*>(a.chi)[a.out_chi_idx] = p;
        if (a.flops) atomicAdd(a.flops, flops);
    }
}

template <class T>
size_t rook_smem_bytes(int kcap) {
    size_t b = sizeof(T) * (2 * (size_t)kcap + RKT);
    b = (b + 15) & ~(size_t)15;
    b += sizeof(RkCand<T>) * (RKT / 32 + 1);
    b = (b + 15) & ~(size_t)15;
    b += sizeof(Decision<T>) + 16;
    return b;
}

template <class T>
size_t creg_bytes(int mmax, int C, int wmax) {
    size_t b = sizeof(T) * (2 * (size_t)mmax + wmax);
    b = (b + 15) & ~(size_t)15;
    b += sizeof(Cand<T>) * (2 * (size_t)C + RWARP) + sizeof(Decision<T>);
    return b;
}

constexpr size_t kSmemLimit = 200 * 1024;

template <class T>
size_t layout_bytes(int mmax, int G, int wcap_elems, int wcap_cols, bool smemw) {
    size_t b = sizeof(T) * ((smemw ? (size_t)wcap_elems : 0) + mmax + wcap_cols + G);
    b = (b + 15) & ~(size_t)15;
    b += sizeof(Decision<T>);
    b += sizeof(unsigned long long) * (NWARP + 1) + sizeof(int) * (NWARP + 1) + sizeof(int) * 4;
    b += (size_t)mmax + (size_t)wcap_cols;
    return (b + 15) & ~(size_t)15;
}

}  // namespace

// Target entries per CTA; ACI_PRRLU_EPC overrides it (launch-shape tuning only).
int prrlu_epc() {
    static const int v = [] {
        const char* e = std::getenv("ACI_PRRLU_EPC");
        const int x = e ? std::atoi(e) : 0;
        return x > 0 ? x : kPrrluEpc;
    }();
    return v;
}

int prrlu_grid(int mmax, int nmax, int num_sms) {
    return live_ctas((long long)mmax * nmax, nmax, std::min(num_sms, PT), prrlu_epc());
}

int prrlu_rook_grid(int mmax, int nmax, int num_sms) {
    const int blocks = std::max((mmax + RKB - 1) / RKB, (nmax + RKB - 1) / RKB);
    return std::max(1, std::min(blocks, num_sms));
}

size_t prrlu_rook_ll_words(int G) { return (size_t)RK_AREAS * G * RK_REC; }

size_t prrlu_rook_scratch_elems(int mmax, int nmax, bool cplx_values) {
    const size_t vb = cplx_values ? 16 : 8;
    return 2 * (size_t)mmax + 2 * (size_t)nmax + ((size_t)mmax + nmax + vb - 1) / vb;
}

size_t prrlu_ll_words(int mmax, int G, bool cplx_values) {
    const int wpv = cplx_values ? 4 : 2;
    return 2 * (size_t)G * kRecWords + 2 * (size_t)G * mmax * wpv;
}

// Shared-memory bytes of the cluster kernel.
template <class T>
size_t cluster_bytes(int mmax, int C, int wcap_elems, int wcap_cols, bool smemw) {
    size_t b = sizeof(T) * ((smemw ? (size_t)wcap_elems : 0) + mmax + wcap_cols);
    b = (b + 15) & ~(size_t)15;
    b += sizeof(Cand<T>) * (2 * (size_t)C + NWARP + 1) + sizeof(Decision<T>);
    b += (size_t)mmax + (size_t)wcap_cols;
    return (b + 15) & ~(size_t)15;
}

// Largest cluster (16, else 8) the device can schedule for the cluster kernel.
template <class T>
int max_cluster_query() {
    int v = 8;
    auto fn = prrlu_cluster_kernel<T, true>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(PT);
        cfg.dynamicSmemBytes = kSmemLimit;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, (void*)fn, &cfg) == cudaSuccess && n >= 1) v = 16;
    }
    cudaGetLastError();
    return v;
}
template <class T>
int max_cluster() {
    static const int v = max_cluster_query<T>();  // once, thread-safe (concurrent batch workers)
    return v;
}

// Shared-memory and cluster-size attributes of a kernel, set once per kernel (host calls such as
// these cost microseconds and would otherwise sit between short launches).
cudaError_t kernel_attrs(const void* fn) {
    static std::mutex mu;
    static std::set<const void*> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(fn)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) cudaGetLastError();  // kernels launched without clusters do not need it
    done.insert(fn);
    return cudaSuccess;
}

// Blocks whose FP64 update work (entries, x4 for complex) is at most this run in one cluster.
constexpr long long kClusterWorkMax = 1LL << 18;
constexpr int kCregColsPerCta = 4;

// ACI_PRRLU_CLUSTER: the cluster size of the single-cluster variants (launch-shape tuning only).
int prrlu_cluster_override() {
    static const int v = [] {
        const char* e = std::getenv("ACI_PRRLU_CLUSTER");
        return e ? std::max(0, std::atoi(e)) : 0;
    }();
    return v;
}

// Live blocks of at most this many entries go to the single-CTA kernel; ACI_PRRLU_SMALL overrides
// it (0 turns the single-CTA kernel off; launch-shape tuning only: the pivots do not depend on it).
constexpr int kPrrluSmallElems = 4096;
int prrlu_small_elems() {
    static const int v = [] {
        const char* e = std::getenv("ACI_PRRLU_SMALL");
        return e ? std::max(0, std::atoi(e)) : kPrrluSmallElems;
    }();
    return v;
}

// The 2D variant for RR rows per lane and CC columns per warp (values per thread: RR CC <= 32
// real, <= 16 complex); nullptr where there is no instantiation.
template <class T>
void (*c2d_kernel(int rr, int cc))(PrrluArgs<T>) {
    if (rr == 1) {
        if (cc == 2) return prrlu_c2d_kernel<T, 1, 2>;
        if (cc == 4) return prrlu_c2d_kernel<T, 1, 4>;
        if (cc == 8) return prrlu_c2d_kernel<T, 1, 8>;
    } else if (rr == 2) {
        if (cc == 2) return prrlu_c2d_kernel<T, 2, 2>;
        if (cc == 4) return prrlu_c2d_kernel<T, 2, 4>;
        if constexpr (sizeof(T) == sizeof(double))  // complex: 16 values spill
            if (cc == 8) return prrlu_c2d_kernel<T, 2, 8>;
    } else if (rr == 4) {
        if (cc == 2) return prrlu_c2d_kernel<T, 4, 2>;
        if (cc == 4) return prrlu_c2d_kernel<T, 4, 4>;
        if constexpr (sizeof(T) == sizeof(double))
            if (cc == 8) return prrlu_c2d_kernel<T, 4, 8>;
    }
    return nullptr;
}

// ACI_PRRLU_2D: 1 (default) the 2D variant for the launch shapes it is faster on, 2 wherever it
// fits, 0 nowhere; ACI_PRRLU_GRIDC=q fixes its column-group count (launch-shape tuning only: the
// pivots are the same).
int prrlu_2d_mode() {
    static const int v = [] {
        const char* e = std::getenv("ACI_PRRLU_2D");
        return e ? std::atoi(e) : 1;
    }();
    return v;
}
int prrlu_gridc_override() {
    static const int v = [] {
        const char* e = std::getenv("ACI_PRRLU_GRIDC");
        return e ? std::max(0, std::atoi(e)) : 0;
    }();
    return v;
}

// The 2D variant exchanges candidates through st.async stores and mbarriers (default; 2-4 % per
// launch faster than the cluster barrier, e.g. 96 x 96: 0.225 vs 0.243 ms, 1000 x 200: 0.901 vs
// 0.928 ms); ACI_PRRLU_MBX=0 takes the cluster barrier (launch-shape tuning only: the pivots are
// the same).
int prrlu_mbx_mode() {
    static const int v = [] {
        const char* e = std::getenv("ACI_PRRLU_MBX");
        return e ? (std::atoi(e) != 0 ? 1 : 0) : 1;
    }();
    return v;
}

// Pivot-search launches of the cluster and single-CTA variants carry the programmatic-serialization
// attribute (the kernel's launch overlaps the end of the previous kernel of the stream, the gather;
// it waits in grid_dependency_wait before reading); ACI_PDL=0 turns that off.
int prrlu_pdl_mode() {
    static const int v = [] {
        const char* e = std::getenv("ACI_PDL");
        return e ? (std::atoi(e) != 0 ? 1 : 0) : 1;
    }();
    return v;
}

static int pow2_at_least(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// The 2D variant's grid for the capacity: Cr x Cc <= cmax CTAs and the per-thread tile (RR, CC)
// minimising a per-step cost in cycles (the FP64 update of a full tile: 4 warps per sub-partition,
// ~64 cycles per warp-wide multiply-add, x4 for complex; the busiest sender's bytes at ~32 bytes
// per clock; ~60 cycles of cluster barrier per CTA). Returns false when no instantiation fits.
template <class T>
bool c2d_plan(int mmax, int nmax, int cmax, int* Cr_out, int* Cc_out, int* rr_out, int* cc_out) {
    const bool cp = sizeof(T) == sizeof(cplx);
    double best = 0.0;
    bool found = false;
    for (int Cr = 1; Cr <= cmax; Cr <<= 1)
        for (int Cc = 1; Cr * Cc <= cmax; Cc <<= 1) {
            if (prrlu_gridc_override() > 0 && Cc != prrlu_gridc_override()) continue;
            if (prrlu_cluster_override() > 0 && Cr * Cc != prrlu_cluster_override()) continue;
            const int rows = (mmax + Cr - 1) / Cr, cols = (nmax + Cc - 1) / Cc;
            const int rr = pow2_at_least((rows + 31) / 32);
            const int cc = std::max(2, pow2_at_least((cols + DWARP - 1) / DWARP));
            if (!c2d_kernel<T>(rr, cc)) continue;
            const double upd = 256.0 * rr * cc * (cp ? 4.0 : 1.0);
            const double xch = ((double)Cc * rows + (double)Cr * cols) * sizeof(T) / 32.0;
            const double cost = upd + xch + 60.0 * Cr * Cc;
            if (!found || cost < best) {
                found = true;
                best = cost;
                *Cr_out = Cr;
                *Cc_out = Cc;
                *rr_out = rr;
                *cc_out = cc;
            }
        }
    return found;
}

// The single-CTA kernel for capacities up to 32 ROWS x 8 W (ROWS rows per lane, W columns per warp).
template <class T>
void (*cta_kernel(int rows, int w))(PrrluArgs<T>) {
    const bool cp = sizeof(T) == sizeof(cplx);
    if (rows == 1) {
        if (w == 4) return prrlu_cta_kernel<T, 1, 4>;
        if (w == 8) return prrlu_cta_kernel<T, 1, 8>;
        return prrlu_cta_kernel<T, 1, 16>;
    }
    if (rows == 2) {
        if (w == 4) return prrlu_cta_kernel<T, 2, 4>;
        if (w == 8) return prrlu_cta_kernel<T, 2, 8>;
        return prrlu_cta_kernel<T, 2, 16>;
    }
    if (!cp) {
        if constexpr (sizeof(T) == sizeof(double)) {
            if (w == 4) return prrlu_cta_kernel<T, 4, 4>;
            if (w == 8) return prrlu_cta_kernel<T, 4, 8>;
            return prrlu_cta_kernel<T, 4, 16>;
        }
    }
    return nullptr;
}

// Launch the single-CTA kernel when its capacity covers the launch's (PrrluArgs::small_*); *covers
// tells whether it did.
template <class T>
cudaError_t launch_small(PrrluArgs<T>& a, cudaStream_t st, bool* covers) {
    *covers = false;
    a.small_m = a.small_n = a.small_elems = 0;
    const int thr = prrlu_small_elems();
    if (thr <= 0) return cudaSuccess;
    const bool cp = sizeof(T) == sizeof(cplx);
    const int mrows = std::min(a.mmax, cp ? 64 : 128), ncols = std::min(a.nmax, 128);
    const int rows = mrows <= 32 ? 1 : (mrows <= 64 ? 2 : 4);
    const int w = ncols <= 32 ? 4 : (ncols <= 64 ? 8 : 16);
    void (*fn)(PrrluArgs<T>) = cta_kernel<T>(rows, w);
    if (!fn) return cudaSuccess;
    // Only when the kernel covers every live shape of the capacity: a second, gated launch per
    // pivot search costs more (several microseconds of launch latency) than it saves.
    if (!(a.mmax <= 32 * rows && a.nmax <= CWARP * w && (long long)a.mmax * a.nmax <= thr)) return cudaSuccess;
    a.small_m = 32 * rows;
    a.small_n = CWARP * w;
    a.small_elems = thr;
    *covers = true;
    cudaError_t e = kernel_attrs((const void*)fn);
    if (e != cudaSuccess) return e;
    size_t smem = sizeof(T) * (2 * 32 * (size_t)rows + 2 * (size_t)CWARP * w + 2);
    smem = ((smem + 15) & ~(size_t)15) + sizeof(Cand<T>) * 2 * CWARP;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(CT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = prrlu_pdl_mode();
    return cudaLaunchKernelEx(&cfg, fn, a);
}

template <class T>
cudaError_t launch_prrlu(const PrrluArgs<T>& a_in, int G, cudaStream_t st) {
    PrrluArgs<T> a = a_in;
    const bool cp = sizeof(T) == sizeof(cplx);
    a.small_m = a.small_n = a.small_elems = 0;
    if (!a.rook) {  // small live blocks: the single-CTA kernel (the others return at once for them)
        bool covers = false;
        cudaError_t e = launch_small<T>(a, st, &covers);
        if (e != cudaSuccess || covers) return e;
    }
    if (a.rook) {
        // the caller sized W (prrlu_rook_scratch_elems), ll (prrlu_rook_ll_words(G)) and gives L, U
        const int kcap = std::max(1, std::min(std::min(a.mmax, a.nmax), a.chimax));
        const size_t smem = rook_smem_bytes<T>(kcap);
        if (smem > kSmemLimit || !a.L || !a.U) return cudaErrorInvalidValue;
        a.wcap_cols = kcap;
        auto fn = prrlu_rook_kernel<T>;
        cudaError_t e = kernel_attrs((const void*)fn);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(G);
        cfg.blockDim = dim3(RKT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, fn, a);
    }
    const long long work = (long long)a.mmax * a.nmax * (cp ? 4 : 1);
    if (work <= kClusterWorkMax || a.no_coop) {  // no_coop: a single cluster at every size
        const int cmax = max_cluster<T>();
        int C = (int)std::min<long long>(cmax, std::max(1LL, (work + 4095) / 4096));
        // At most kCregColsPerCta columns per CTA where the cluster allows: the FP64 units of an SM
        // sub-partition take ~64 cycles per warp-wide multiply-add, so the update of a step costs
        // (row warps per sub-partition) x (columns per CTA) x ~64 cycles, and spreading the columns
        // over more SMs shortens every step more than the wider exchange lengthens it (measured
        // 25-35% per launch from 20 x 20 to 200 x 200).
        C = std::max(C, std::min(cmax, (a.nmax + kCregColsPerCta - 1) / kCregColsPerCta));
        C = std::max(1, std::min(C, a.nmax));
        if (prrlu_cluster_override() > 0) C = std::max(1, std::min(std::min(prrlu_cluster_override(), cmax), a.nmax));
        const int wneed = (a.nmax + C - 1) / C;
        const int rows = (a.mmax + RT - 1) / RT;
        // The 2D variant where it measured faster than the 1D register variant (per launch, GB300):
        // complex blocks, real blocks of more than 512 rows, real blocks whose 1D split leaves at
        // most 8 columns per CTA, and real blocks whose 2D tile holds at most 8 values per thread
        // (256 x 256: 0.476 vs 0.508 ms); the 1D variant keeps the larger real blocks of up to 512
        // rows (480 x 480: 1.36 vs 1.56 ms, 480 x 246: 0.83 vs 0.87). ACI_PRRLU_2D = 2 takes the 2D
        // variant wherever it fits, 0 nowhere.
        int Cr = 0, Cc = 0, rr = 0, cc = 0;
        const bool fits2d = c2d_plan<T>(a.mmax, a.nmax, cmax, &Cr, &Cc, &rr, &cc);
        const bool prefer2d = cp || rows > 1 || wneed <= 8 || rr * cc <= 8;
        if (fits2d && (prrlu_2d_mode() == 2 || (prrlu_2d_mode() == 1 && prefer2d))) {
            void (*fn)(PrrluArgs<T>) = c2d_kernel<T>(rr, cc);
            a.epc = 0;
            a.wcap_cols = cc;
            a.wcap_elems = 0;
            a.grid_c = Cc;
            a.c2d_mbx = prrlu_mbx_mode();
            cudaError_t e = kernel_attrs((const void*)fn);
            if (e != cudaSuccess) return e;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(Cr * Cc);
            cfg.blockDim = dim3(DT);
            cfg.dynamicSmemBytes = c2d_bytes<T>(rr, cc, Cr * Cc);
            cfg.stream = st;
            cudaLaunchAttribute at[2];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = Cr * Cc;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[1].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1 + prrlu_pdl_mode();
            return cudaLaunchKernelEx(&cfg, fn, a);
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C);
        cfg.stream = st;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1 + prrlu_pdl_mode();
        void (*reg)(PrrluArgs<T>) = nullptr;
        int wmax = 0;
        // register budget: at most 32 values per thread (real) or 16 (complex)
        if (rows == 1) {
            if (wneed <= 8) { reg = prrlu_creg_kernel<T, 1, 8>; wmax = 8; }
            else if (wneed <= 16) { reg = prrlu_creg_kernel<T, 1, 16>; wmax = 16; }
            else if constexpr (sizeof(T) == sizeof(double)) {
                if (wneed <= 32) { reg = prrlu_creg_kernel<T, 1, 32>; wmax = 32; }
            }
        } else if (rows == 2) {
            if (wneed <= 8) { reg = prrlu_creg_kernel<T, 2, 8>; wmax = 8; }
            else if constexpr (sizeof(T) == sizeof(double)) {
                if (wneed <= 16) { reg = prrlu_creg_kernel<T, 2, 16>; wmax = 16; }
            }
        }
        if (reg) {
            a.epc = 0;
            a.wcap_cols = wmax;
            a.wcap_elems = 0;
            const size_t smem = creg_bytes<T>(a.mmax, C, wmax);
            cudaError_t e = kernel_attrs((const void*)reg);
            if (e != cudaSuccess) return e;
            cfg.blockDim = dim3(RT);
            cfg.dynamicSmemBytes = smem;
            return cudaLaunchKernelEx(&cfg, reg, a);
        }
        a.epc = 0;
        a.wcap_cols = wneed;
        a.wcap_elems = a.mmax * a.wcap_cols;
        const bool smemw = cluster_bytes<T>(a.mmax, C, a.wcap_elems, a.wcap_cols, true) <= kSmemLimit;
        const size_t smem = cluster_bytes<T>(a.mmax, C, a.wcap_elems, a.wcap_cols, smemw);
        if (smem > kSmemLimit) return cudaErrorInvalidValue;
        void (*fn)(PrrluArgs<T>) = smemw ? prrlu_cluster_kernel<T, true> : prrlu_cluster_kernel<T, false>;
        cudaError_t e = kernel_attrs((const void*)fn);
        if (e != cudaSuccess) return e;
        cfg.blockDim = dim3(PT);
        cfg.dynamicSmemBytes = smem;
        return cudaLaunchKernelEx(&cfg, fn, a);
    }
    a.epc = prrlu_epc();
    // worst-case block over every live shape this launch may meet (see live_ctas)
    const int ceil_n = (a.nmax + G - 1) / G;
    a.wcap_elems = std::max(a.epc + a.mmax, a.mmax * ceil_n);
    a.wcap_cols = std::min(a.nmax, std::max(ceil_n, a.epc));
    const bool smemw = layout_bytes<T>(a.mmax, G, a.wcap_elems, a.wcap_cols, true) <= kSmemLimit;
    const size_t smem = layout_bytes<T>(a.mmax, G, a.wcap_elems, a.wcap_cols, smemw);
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    void (*fn)(PrrluArgs<T>) = smemw ? prrlu_kernel<T, true> : prrlu_kernel<T, false>;
    cudaError_t e = kernel_attrs((const void*)fn);
    if (e != cudaSuccess) return e;
    // a cooperative launch (all CTAs co-resident), expressed so that stream capture accepts it
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(PT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

namespace {
__global__ void recip_kernel(const double* x, int n, double* y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = recip_of(x[i]);
}
}  // namespace

void launch_recip(const double* x, int n, double* y, cudaStream_t st) {
    if (n > 0) recip_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, n, y);
}

template cudaError_t launch_prrlu<double>(const PrrluArgs<double>&, int, cudaStream_t);
template cudaError_t launch_prrlu<cplx>(const PrrluArgs<cplx>&, int, cudaStream_t);

}  // namespace aci
