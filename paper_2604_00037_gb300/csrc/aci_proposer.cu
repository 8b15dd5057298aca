// The learned proposer's device side (not in the paper): candidate features of a Pi block, the
// top-K selection that restricts the block, the map of the restricted pivots back to Pi, and the
// recording of (features, pivot-or-not) pairs for training.
//
// Candidates of bond b are the rows r = alpha d_b + sigma of Pi (alpha < chi_b) and its columns
// c = sigma' chi_{b+2} + beta. Features (kPropFeatures = 7), in [-2, 1]:
//   0, 1  log2 of the candidate's norm in the first / second input's environment (row of the
//         Pi-A operand, column of the Pi-B operand), minus the largest over the bond's candidates
//         of the same side, over 32 (clipped at -2);
//   2     sigma / (d - 1);  3  alpha / chi (position of the parent pivot);  4  b / (L - 1);
//   5     1 if the candidate was a pivot of this bond in the previous sweep;  6  1 for columns.
#include <algorithm>
#include <climits>
#include <mutex>

#include "aci_internal.h"

namespace aci {

namespace {

constexpr int kPT = 1024;

__device__ __forceinline__ double sq(double v) { return v * v; }
__device__ __forceinline__ double sq(cplx v) { return v.re * v.re + v.im * v.im; }

// Order-preserving int image of a float (for atomicMax) and its inverse.
__device__ __forceinline__ int fkey(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float fkey_inv(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7FFFFFFF); }

constexpr int kNT = 256;  // threads of the norm kernel

// Pass 1 over the whole GPU: 0.5 log2 of each candidate's squared norm per input, into features 0
// and 1 (raw), and the side maxima. Rows: one warp per row (lanes along K, coalesced); columns: one
// thread per column (threads along the row of B, coalesced).
template <class T>
__global__ void __launch_bounds__(kNT) features_norm_kernel(ProposerArgs<T> a, int row_blocks) {
    const int lane = threadIdx.x & 31;
    const bool cols = (int)blockIdx.x >= row_blocks;
    float l2[2] = {-1e30f, -1e30f};
    int i;
    bool valid;
    if (!cols) {
        i = (int)blockIdx.x * (kNT / 32) + (threadIdx.x >> 5);
        valid = i < dimv(a.M, a.chi);
        if (i >= a.mcap) return;  // whole warp
        for (int q = 0; q < a.nprod; ++q) {
            double s = 0.0;
            if (valid) {
                const int K = dimv(a.K[q], a.chi), lda = dimv(a.lda[q], a.chi);
                const T* row = a.A[q] + (size_t)i * lda;
                for (int k = lane; k < K; k += 32) s += sq(row[k]);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            l2[q] = s > 0.0 ? 0.5f * log2f((float)s) : -1e30f;
        }
        if (lane != 0) return;
    } else {
        i = ((int)blockIdx.x - row_blocks) * kNT + threadIdx.x;
        if (i >= a.ncap) return;
        valid = i < dimv(a.N, a.chi);
        for (int q = 0; q < a.nprod && valid; ++q) {
            const int K = dimv(a.K[q], a.chi), ldb = dimv(a.ldb[q], a.chi);
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += sq(a.B[q][(size_t)k * ldb + i]);
            l2[q] = s > 0.0 ? 0.5f * log2f((float)s) : -1e30f;
        }
    }
    if (a.nprod == 1) l2[1] = l2[0];
    float* x = a.X + ((cols ? (size_t)a.mcap : 0) + i) * kPropFeatures;
    x[0] = l2[0];
    x[1] = l2[1];
    if (valid) {
        atomicMax(a.side_max + (cols ? 2 : 0), fkey(l2[0]));
        atomicMax(a.side_max + (cols ? 3 : 1), fkey(l2[1]));
    }
}

// Pass 2, one CTA per side: features 0 and 1 relative to the side maxima, the others from the
// candidate's position; resets the side maxima for the next call.
template <class T>
__global__ void __launch_bounds__(kPT) features_kernel(ProposerArgs<T> a) {
    constexpr int kBits = 1 << 16;  // previous-pivot bitmap (larger sides scan the list instead)
    __shared__ unsigned int was_bits[kBits / 32];
    const bool cols = blockIdx.x == 1;
    const int live = cols ? dimv(a.N, a.chi) : dimv(a.M, a.chi);
    const int cap = cols ? a.ncap : a.mcap;
    const int dloc = cols ? a.d_col : a.d_row;
    const int chi_side = cols ? dimv(a.chi_col, a.chi) : dimv(a.chi_row, a.chi);
    const int kprev = dimv(a.kprev, a.chi);
    const int* prev = cols ? a.prev_cols : a.prev_rows;
    float* X = a.X + (cols ? (size_t)a.mcap * kPropFeatures : 0);
    int* smx = a.side_max + (cols ? 2 : 0);
    const float lmax[2] = {fkey_inv(smx[0]), fkey_inv(smx[1])};
    const bool bitmap = cap <= kBits;
    if (bitmap) {
        for (int w = threadIdx.x; w < (cap + 31) / 32; w += kPT) was_bits[w] = 0u;
        __syncthreads();
        for (int p = threadIdx.x; p < kprev; p += kPT) {
            const int r = prev[p];
            if (r >= 0 && r < cap) atomicOr(&was_bits[r >> 5], 1u << (r & 31));
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < cap; i += kPT) {
        float* x = X + (size_t)i * kPropFeatures;
        if (i >= live) {
            for (int f = 0; f < kPropFeatures; ++f) x[f] = 0.f;
            continue;
        }
        for (int q = 0; q < 2; ++q) x[q] = fmaxf((x[q] - lmax[q]) / 32.f, -2.f);
        const int sigma = cols ? i / max(chi_side, 1) : i % dloc;
        const int pos = cols ? i % max(chi_side, 1) : i / dloc;
        x[2] = dloc > 1 ? (float)sigma / (float)(dloc - 1) : 0.f;
        x[3] = (float)pos / (float)max(chi_side, 1);
        x[4] = a.bond_frac;
        int was = 0;
        if (bitmap) {
            was = (was_bits[i >> 5] >> (i & 31)) & 1u;
        } else {
            for (int p = 0; p < kprev; ++p) was |= prev[p] == i;
        }
        x[5] = (float)was;
        x[6] = cols ? 1.f : 0.f;
    }
    __syncthreads();
    if (threadIdx.x < 2) smx[threadIdx.x] = INT_MIN;
}

// Keep the K best-scoring live candidates of each side, in ascending index order; K = min(live,
// ceil(keep * kprev) + 8). Block 0 rows, block 1 columns; bitonic sort of (score, index) in
// shared memory (ties: lower index first).
__global__ void __launch_bounds__(kPT) topk_kernel(TopkArgs t) {
    extern __shared__ unsigned char sm[];
    const bool cols = blockIdx.x == 1;
    const int live = cols ? dimv(t.N, t.chi) : dimv(t.M, t.chi);
    const int cap = cols ? t.ncap : t.mcap;
    const float* z = t.z + (cols ? t.mcap : 0);
    int P = 1;
    while (P < cap) P <<= 1;
    float* key = reinterpret_cast<float*>(sm);
    int* idx = reinterpret_cast<int*>(key + P);
    int* flag = idx + P;
    for (int i = threadIdx.x; i < P; i += kPT) {
        key[i] = i < live ? z[i] : -INFINITY;
        idx[i] = i;
        if (i < cap) flag[i] = 0;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += kPT) {
                const int l = i ^ j;
                if (l > i) {
                    // descending by key, ascending by index
                    const bool before = key[i] > key[l] || (key[i] == key[l] && idx[i] < idx[l]);
                    const bool up = (i & k) == 0;
                    if (up != before) {
                        const float kt = key[i]; key[i] = key[l]; key[l] = kt;
                        const int it = idx[i]; idx[i] = idx[l]; idx[l] = it;
                    }
                }
            }
            __syncthreads();
        }
    const int kprev = dimv(t.kprev, t.chi);
    int K = (int)ceilf(t.keep * (float)kprev) + 8;
    K = min(K, live);
    K = max(K, min(live, 1));
    for (int i = threadIdx.x; i < K; i += kPT) flag[idx[i]] = 1;
    __syncthreads();
    // ascending compaction of the flags (one thread: cap <= a few thousand)
    if (threadIdx.x == 0) {
        int* sel = cols ? t.sel_cols : t.sel_rows;
        int o = 0;
        for (int i = 0; i < cap; ++i)
            if (flag[i]) sel[o++] = i;
        const_cast<int*>(t.chi)[cols ? t.slot_cols : t.slot_rows] = K;
    }
}

// prow[p] = sel_rows[prow[p]], pcol[p] = sel_cols[pcol[p]] for p < k
__global__ void map_pivots_kernel(const int* chi, int kslot, int* prow, int* pcol, const int* sel_rows,
                                  const int* sel_cols) {
    const int k = chi[kslot];
    for (int p = threadIdx.x; p < k; p += blockDim.x) {
        prow[p] = sel_rows[prow[p]];
        pcol[p] = sel_cols[pcol[p]];
    }
}

// Append (features, 1 if a pivot of the new sets else 0) for every live candidate of the bond.
__global__ void record_kernel(RecordArgs r) {
    const int m = dimv(r.M, r.chi), n = dimv(r.N, r.chi), k = dimv(r.k, r.chi);
    const int total = m + n;
    __shared__ long long base;
    if (threadIdx.x == 0) {
        base = (long long)atomicAdd(r.count, (unsigned long long)total);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const long long o = base + i;
        if (o >= r.capacity) break;
        const bool col = i >= m;
        const int c = col ? i - m : i;
        const float* x = r.X + (size_t)(col ? r.mcap + c : c) * kPropFeatures;
        const int* piv = col ? r.pcol : r.prow;
        int lab = 0;
        for (int p = 0; p < k; ++p) lab |= piv[p] == c;
        float* out = r.buf + (size_t)o * (kPropFeatures + 1);
        for (int f = 0; f < kPropFeatures; ++f) out[f] = x[f];
        out[kPropFeatures] = (float)lab;
    }
}

}  // namespace

template <class T>
void launch_features(const ProposerArgs<T>& a, cudaStream_t st) {
    const int row_blocks = (a.mcap + kNT / 32 - 1) / (kNT / 32);
    const int col_blocks = (a.ncap + kNT - 1) / kNT;
    features_norm_kernel<T><<<row_blocks + col_blocks, kNT, 0, st>>>(a, row_blocks);
    features_kernel<T><<<2, kPT, 0, st>>>(a);
}
template void launch_features<double>(const ProposerArgs<double>&, cudaStream_t);
template void launch_features<cplx>(const ProposerArgs<cplx>&, cudaStream_t);

size_t topk_smem(int mcap, int ncap) {
    int P = 1;
    while (P < std::max(mcap, ncap)) P <<= 1;
    return (size_t)P * (sizeof(float) + 2 * sizeof(int));
}

cudaError_t launch_topk(const TopkArgs& t, cudaStream_t st) {
    const size_t smem = topk_smem(t.mcap, t.ncap);
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (attr != cudaSuccess) return attr;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    topk_kernel<<<2, kPT, smem, st>>>(t);
    return cudaGetLastError();
}

void launch_map_pivots(const int* chi, int kslot, int* prow, int* pcol, const int* sel_rows, const int* sel_cols,
                       cudaStream_t st) {
    map_pivots_kernel<<<1, 256, 0, st>>>(chi, kslot, prow, pcol, sel_rows, sel_cols);
}

void launch_record(const RecordArgs& r, cudaStream_t st) { record_kernel<<<1, 1024, 0, st>>>(r); }

}  // namespace aci
