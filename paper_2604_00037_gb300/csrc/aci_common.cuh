// Shared device definitions of the ACI library: scalar types, the elementwise function f,
// the pivot key, and the descriptors through which kernels read shapes that are only known
// on the device (the ranks chosen by earlier pivot searches).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace aci {

// Interleaved complex128, 16-byte aligned so a value moves as one double2.
struct __align__(16) cplx {
    double re, im;
};

__host__ __device__ inline cplx mkc(double r, double i) { cplx z; z.re = r; z.im = i; return z; }

// ---------------------------------------------------------------- scalar arithmetic
// Real and complex versions of the few operations the kernels need.
__device__ __forceinline__ double s_zero(double) { return 0.0; }
__device__ __forceinline__ cplx s_zero(cplx) { return mkc(0.0, 0.0); }
__device__ __forceinline__ double s_one(double) { return 1.0; }
__device__ __forceinline__ cplx s_one(cplx) { return mkc(1.0, 0.0); }

__device__ __forceinline__ double s_add(double a, double b) { return a + b; }
__device__ __forceinline__ cplx s_add(cplx a, cplx b) { return mkc(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ double s_mul(double a, double b) { return a * b; }
// The complex product with its fused multiply-adds written out: left to the compiler, which of
// the two products it fuses may differ from kernel to kernel, and so would the rounding.
__device__ __forceinline__ cplx s_mul(cplx a, cplx b) {
    return mkc(fma(a.re, b.re, -__dmul_rn(a.im, b.im)), fma(a.re, b.im, __dmul_rn(a.im, b.re)));
}
// acc + a * b
__device__ __forceinline__ double s_fma(double a, double b, double acc) { return fma(a, b, acc); }
__device__ __forceinline__ cplx s_fma(cplx a, cplx b, cplx acc) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
    return acc;
}
// acc - a * b
__device__ __forceinline__ double s_fms(double a, double b, double acc) { return fma(-a, b, acc); }
__device__ __forceinline__ cplx s_fms(cplx a, cplx b, cplx acc) {
    acc.re = fma(-a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(-a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
    return acc;
}
__device__ __forceinline__ double s_conj(double a) { return a; }
__device__ __forceinline__ cplx s_conj(cplx a) { return mkc(a.re, -a.im); }
__device__ __forceinline__ double s_div(double a, double b) { return a / b; }
__device__ __forceinline__ cplx s_div(cplx a, cplx b) {
    // Smith's algorithm (R. L. Smith, CACM 1962) to avoid overflow in |b|^2.
    // (fused multiply-adds written out, as in s_mul)
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, den = fma(b.im, r, b.re);
        return mkc(fma(a.im, r, a.re) / den, fma(-a.re, r, a.im) / den);
    } else {
        const double r = b.re / b.im, den = fma(b.re, r, b.im);
        return mkc(fma(a.re, r, a.im) / den, fma(a.im, r, -a.re) / den);
    }
}
__device__ __forceinline__ bool s_iszero(double a) { return a == 0.0; }
__device__ __forceinline__ bool s_iszero(cplx a) { return a.re == 0.0 && a.im == 0.0; }
__device__ __forceinline__ bool s_finite(double a) { return isfinite(a); }
__device__ __forceinline__ bool s_finite(cplx a) { return isfinite(a.re) && isfinite(a.im); }

// Pivot key maximised by the pivot search: |v| for real, re*re + im*im for complex, each
// product and the sum rounded separately (no fused multiply-add) so the CPU oracle
// computes bit-identical keys from identical values.
__device__ __forceinline__ double s_key(double a) { return fabs(a); }
__device__ __forceinline__ double s_key(cplx a) { return __dadd_rn(__dmul_rn(a.re, a.re), __dmul_rn(a.im, a.im)); }
// |v| (sqrt is correctly rounded).
__device__ __forceinline__ double s_mag(double a) { return fabs(a); }
__device__ __forceinline__ double s_mag(cplx a) { return __dsqrt_rn(s_key(a)); }
__device__ __forceinline__ double key_to_mag(double k, double) { return k; }
__device__ __forceinline__ double key_to_mag(double k, cplx) { return __dsqrt_rn(k); }

// Bits of the pivot key of a value. Keys are non-negative doubles, which order like their bit
// patterns, so maxima are taken on 64-bit integers (the FP64 pipe is scarce on GB300). For real
// values the key |v| is formed by clearing the sign bit: bit-identical to fabs, no FP64 op.
__device__ __forceinline__ unsigned long long key_of(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    // an explicit integer AND: left to itself the compiler turns the mask back into fabs,
    // which on this GPU costs an FP64 operation per entry
    asm("and.b64 %0, %0, 0x7FFFFFFFFFFFFFFF;" : "+l"(b));
    return b;
}
__device__ __forceinline__ unsigned long long key_of(cplx v) {
    return (unsigned long long)__double_as_longlong(s_key(v));
}

// |a|^2 a (the oracle computes (a*a)*a for real and (re*re + im*im) * a for complex).
__device__ __forceinline__ double abs2_mul(double a) { return (a * a) * a; }
__device__ __forceinline__ cplx abs2_mul(cplx a) {
    double n2 = __dadd_rn(__dmul_rn(a.re, a.re), __dmul_rn(a.im, a.im));
    return mkc(n2 * a.re, n2 * a.im);
}

template <class T> struct dtype_id;
template <> struct dtype_id<double> { static constexpr int value = 0; };
template <> struct dtype_id<cplx> { static constexpr int value = 1; };

// ---------------------------------------------------------------- elementwise f (Sec. 2.1)
enum OpKind { OP_MUL = 0, OP_MUL_CONJ = 1, OP_ABS2_MUL = 2, OP_AFFINE = 3 };

template <class T> struct OpParams {
    int kind;
    T c[4];
};

// f applied to the N = 1 or 2 products at one entry; matches the oracle's expression order.
template <class T>
__device__ __forceinline__ T apply_f(const OpParams<T>& op, T a, T b) {
    switch (op.kind) {
        case OP_MUL: return s_mul(a, b);
        case OP_MUL_CONJ: return s_mul(a, s_conj(b));
        case OP_ABS2_MUL: return abs2_mul(a);
        default: {
            T r = op.c[0];
            r = s_add(r, s_mul(op.c[1], a));
            r = s_add(r, s_mul(op.c[2], b));
            r = s_add(r, s_mul(op.c[3], s_mul(a, b)));
            return r;
        }
    }
}

// f of n inputs (n >= 1): apply_f for n <= 2; for more inputs the library's only op is the
// product of all of them, formed left to right as the oracle does.
constexpr int kMaxInputs = 4;
template <class T>
__device__ __forceinline__ T apply_fn(const OpParams<T>& op, const T* v, int n) {
    if (n <= 2) return apply_f(op, v[0], n > 1 ? v[1] : v[0]);
    T r = s_mul(v[0], v[1]);
    for (int i = 2; i < n; ++i) r = s_mul(r, v[i]);
    return r;
}

// ---------------------------------------------------------------- device-resolved shapes
// A dimension that depends on the ranks chosen on the device: value = mul * chi[idx]
// (or mul when idx < 0). chi[] is the device array of output ranks chi[0..L].
struct DimE {
    int mul;
    int idx;
};
__host__ __device__ inline DimE dimc(int v) { DimE e; e.mul = v; e.idx = -1; return e; }
__host__ __device__ inline DimE dimr(int mul, int idx) { DimE e; e.mul = mul; e.idx = idx; return e; }
__device__ __forceinline__ int dimv(DimE e, const int* chi) { return e.idx >= 0 ? e.mul * chi[e.idx] : e.mul; }

// Index maps of the gathers. Row r: none (idx NULL), plain (blk 0: idx[r]) or by blocks of blk
// rows (idx[r / blk] * blk + r % blk: rows idx of a matrix whose rows are blk rows long each).
// Column c: none, plain (blk 0: idx[c]) or by blocks of blk columns, each block taken from a slab
// of `stride` source columns (c / blk * stride + idx[c % blk]).
__device__ __forceinline__ int gather_row(const int* idx, int blk, int r) {
    if (!idx) return r;
    return blk > 0 ? idx[r / blk] * blk + r % blk : idx[r];
}
__device__ __forceinline__ int gather_col(const int* idx, int blk, int stride, int c) {
    if (!idx) return c;
    return blk > 0 ? (c / blk) * stride + idx[c % blk] : idx[c];
}

// Error flags raised by kernels and read by the host once per sweep.
enum DevErr { DEVERR_TIMEOUT = 1, DEVERR_NUMERIC = 2 };

// Iteration limit of every device-side wait (about a second of polling).
constexpr long long kSpinLimit = 1LL << 24;

}  // namespace aci

