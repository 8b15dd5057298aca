// Tensor-core form of the ACI contractions: the frame half-products (Algorithm 5) and the Pi block
// with f in the epilogue (Eq. (pifromframes), Eq. (localupdate)), the same operands and results as
// gemm_kernel, computed on the 5th-generation tensor cores (tcgen05) from exact BF16 digit planes.
//
// FP64 has no tcgen05 kind, so every FP64 operand is cut into S digit planes that BF16 holds
// exactly (the error-free splitting of Ozaki, Ogita, Oishi and Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication and its applications",
// Numer. Algorithms 59 (2012)). Row r of A gets the scale 2^e_r, the smallest power of two above
// max_k |A[r,k]|, column c of B the scale 2^f_c; the scaled values are truncated to S digits of b
// bits, a_i in [-(2^b - 1), 2^b - 1], most significant first:
//   A[r,k] ~ 2^e_r  sum_{i<S} a_i[r,k] 2^(-b(i+1)),    B[k,c] ~ 2^f_c  sum_{j<S} b_j[k,c] 2^(-b(j+1)).
// The digit products of order t = i + j (t < S are kept) are summed over k into one FP32
// accumulator per order in tensor memory. b is chosen so that S K (2^b - 1)^2 < 2^24, so every
// partial sum is an integer FP32 holds exactly. The epilogue forms
//   C[r,c] = 2^(e_r + f_c - b(S+1)) sum_{t<S} acc_t[r,c] 2^(b(S-1-t))
// in integers (two int64 halves, one rounding into FP64). Per element,
//   |C - C_exact| <= K 2^(e_r + f_c) 2^(-bS) (S + 3.1)   (operand truncation plus dropped orders).
//
// Complex operands run as one real product of twice the size: A viewed as M x 2K real (the
// interleaved storage itself), B as the 2K x 2N real matrix [[Re B, Im B], [-Im B, Re B]] (row
// pairs k, column pairs c), whose product is the interleaved complex result.
//
// Kernels. tc_split_kernel writes the digit planes of every operand of a launch straight into the
// shared-memory layout the tensor cores read: per (product, digit, tile) a run of K slabs of 16,
// each slab the no-swizzle K-major arrangement of 8 x 16-byte core matrices (8-row groups 128 bytes
// apart, the two 8-wide K halves R*16 bytes apart for a tile of R rows). tc_gemm_kernel (one
// 128-row x NT-column output tile per CTA, 128 threads) runs a ring of stages: one thread issues
// the bulk copies (cp.async.bulk with mbarrier transaction counts), one thread issues tcgen05.mma for
// every digit pair into the order's accumulator, tcgen05.commit frees a stage when the MMAs reading
// it are done, and all four warps read the accumulators back with tcgen05.ld for the epilogue
// (recombination, f, store, running maximum). Every wait is bounded in time; on a timeout the
// kernel records DEVERR_TIMEOUT, waits (bounded) for its copies in flight and releases tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include <cstdlib>

#include "aci_internal.h"

namespace aci {

namespace {

constexpr int kTileM = 128;                  // rows per output tile (tcgen05 M)
constexpr int kSlabK = 16;                   // K per slab (tcgen05 K for 16-bit inputs)
constexpr int kStageSlabs = 1;               // slabs per pipeline stage
constexpr uint32_t kSlabBytesA = kTileM * kSlabK * 2;  // 4 KB
constexpr int kSplitMaxWarps = 16;  // warps of a split CTA along K (32 rows per CTA)
constexpr int kSplitCache = 2;     // 8-wide K groups a lane keeps in registers between the passes
constexpr int kGemmThreads = 256;  // 8 warps: warps w and w + 4 read the same TMEM lanes, other columns
constexpr int kExpNonFinite = 1 << 20;       // scale marker of a row or column holding Inf or NaN
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory matrix descriptor, no swizzle: start >> 4, K-direction core-matrix stride (LBO) >> 4,
// 8-row-group stride (SBO) >> 4, descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// polls > 0: give up after that many failed polls (a diagnostic limit, aci_set_wait_limits);
// 0: after kWaitNs of polling.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, long long polls = 0) {
    if (mbar_try(bar, parity)) return true;
    if (polls > 0) {
        for (long long it = 1; it < polls; ++it)
            if (mbar_try(bar, parity)) return true;
        return false;
    }
    const unsigned long long t0 = gtimer();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63u) == 0 && gtimer() - t0 > kWaitNs) return false;
    }
}

// ------------------------------------------------------------------ digit split

// Operand values as a real matrix: A'' (rows x K''), B'' read as its transpose (N'' x K'').
__device__ __forceinline__ double a_val(const double* A, int src, int lda, int k) { return A[(size_t)src * lda + k]; }
__device__ __forceinline__ double a_val(const cplx* A, int src, int lda, int k) {
    return reinterpret_cast<const double*>(A)[(size_t)src * 2 * lda + k];
}
__device__ __forceinline__ double b_val(const double* B, int ldb, int col, int n, int k) {
    (void)n;
    return B[(size_t)k * ldb + col];
}
// B'' row 2k + h, column 2c + p: [[Re, Im], [-Im, Re]] of B[k, c]
__device__ __forceinline__ double b_val(const cplx* B, int ldb, int col, int n, int k) {
    const cplx v = B[(size_t)(k >> 1) * ldb + col];
    const int p = n & 1, h = k & 1;
    return p == 0 ? (h == 0 ? v.re : -v.im) : (h == 0 ? v.im : v.re);
}

// floor(|x| 2^(sb - e)) for |x| < 2^e, exactly, from the bits of |x|.
__device__ __forceinline__ unsigned long long scaled_int(unsigned long long xb, int sb, int e) {
    int ex = (int)(xb >> 52);
    unsigned long long man = xb & 0x000FFFFFFFFFFFFFull;
    if (ex == 0) ex = 1;
    else man |= 0x0010000000000000ull;
    const int sh = ex - 1075 + sb - e;
    if (sh >= 0) return man << sh;
    if (sh > -64) return man >> (-sh);
    return 0;
}

// Exact BF16 bits of a small integer v, |v| < 2^8: 1.5 * 2^23 + v is exact in FP32 (ulp 1), the
// subtraction gives (float)v exactly, and its low 16 bits are zero.
__device__ __forceinline__ uint32_t bf16_of_int(int v) {
    const float f = __int_as_float(0x4B400000 + v) - 12582912.0f;
    return __float_as_uint(f) >> 16;
}

template <class T>
__global__ void __launch_bounds__(32 * kSplitMaxWarps) tc_split_kernel(TcArgs<T> a) {
    __shared__ unsigned long long part[kSplitMaxWarps][32];
    const int o = blockIdx.y;
    const int nq = a.nprod;
    if (o >= 2 * nq) return;
    const bool isA = o < nq;
    const int q = isA ? o : o - nq;
    const int z = a.combine ? 0 : q;
    constexpr int cmul = (sizeof(T) == sizeof(cplx)) ? 2 : 1;
    const int rows_live = isA ? dimv(a.M[z], a.chi) : cmul * dimv(a.N[z], a.chi);
    const int tile = isA ? kTileM : a.NT;
    const int rows_fill = (rows_live + tile - 1) / tile * tile;
    if ((int)blockIdx.x * 32 >= rows_fill) return;
    const int W = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * 32 + lane;
    const bool live = r < rows_live;
    const int K2 = cmul * dimv(a.K[q], a.chi);
    const int ngroups = (K2 + kSlabK - 1) / kSlabK * 2;  // 8-wide K groups up to the slab boundary

    int src = 0;  // source row of A, or source column of B
    if (live) {
        if (isA) src = a.arow ? a.arow[r] : r;
        else {
            const int c = r / cmul;
            src = a.bcol ? a.bcol[c] : c;
        }
    }
    const T* Aq = a.A[q];
    const T* Bq = a.B[q];
    const int lda = dimv(a.lda[q], a.chi), ldb = dimv(a.ldb[q], a.chi);
    auto load = [&](int k) -> unsigned long long {
        if (!live || k >= K2) return 0ull;
        const double x = isA ? a_val(Aq, src, lda, k) : b_val(Bq, ldb, src, r, k);
        return (unsigned long long)__double_as_longlong(x);
    };

    // pass 1: the lane's first groups stay in registers; the row maximum over all groups
    unsigned long long xc[kSplitCache][8];
    unsigned long long mb = 0;
#pragma unroll
    for (int gi = 0; gi < kSplitCache; ++gi) {
        const int g = warp + gi * W;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            xc[gi][j] = g < ngroups ? load(8 * g + j) : 0ull;
            const unsigned long long bb = xc[gi][j] & 0x7FFFFFFFFFFFFFFFull;
            mb = bb > mb ? bb : mb;
        }
    }
    for (int g = warp + kSplitCache * W; g < ngroups; g += W)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const unsigned long long bb = load(8 * g + j) & 0x7FFFFFFFFFFFFFFFull;
            mb = bb > mb ? bb : mb;
        }
    part[warp][lane] = mb;
    __syncthreads();
    for (int w = 0; w < W; ++w) mb = part[w][lane] > mb ? part[w][lane] : mb;
    const bool finite = mb < 0x7FF0000000000000ull;
    int e = 0;
    if (mb != 0 && finite) {
        const int ex = (int)(mb >> 52);
        e = ex == 0 ? -1022 : ex - 1022;  // the smallest e with max |x| < 2^e
    }
    if (warp == 0) {
        int* expo = isA ? a.expoA + (size_t)q * a.mtiles * kTileM : a.expoB + (size_t)q * a.ntiles * a.NT;
        expo[r] = finite ? e : kExpNonFinite;
    }
    const int S = a.S, b = a.bits, sb = S * b;
    const unsigned mask = (1u << b) - 1u;
    const int t_idx = r / tile, rr = r % tile;
    // A: [q][mt][slab][digit] blocks of 128 x 16; B: [q][nt][slab] blocks of S*NT x 16, digit i in
    // rows [i*NT, (i+1)*NT). In a block of R rows, K half h starts at h*R*16 bytes.
    const int brows = isA ? kTileM : S * a.NT;
    unsigned char* base = isA ? a.planesA : a.planesB;
    const size_t tile_slab0 = ((size_t)q * (isA ? a.mtiles : a.ntiles) + t_idx) * a.ksl;
    auto emit = [&](int g, const unsigned long long* xb) {
        unsigned long long y[8];
        uint32_t neg = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const unsigned long long v = finite ? xb[j] : 0ull;
            y[j] = scaled_int(v & 0x7FFFFFFFFFFFFFFFull, sb, e);
            neg |= (uint32_t)(v >> 63) << j;
        }
        const size_t slab = tile_slab0 + (g >> 1);
        for (int i = 0; i < S; ++i) {
            const int shift = b * (S - 1 - i);
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int v0 = (int)((y[2 * j] >> shift) & mask), v1 = (int)((y[2 * j + 1] >> shift) & mask);
                if (neg >> (2 * j) & 1) v0 = -v0;
                if (neg >> (2 * j + 1) & 1) v1 = -v1;
                w[j] = bf16_of_int(v0) | (bf16_of_int(v1) << 16);
            }
            size_t off;
            if (isA) {
                off = (slab * S + i) * kSlabBytesA + (uint32_t)(g & 1) * (kTileM * 16) + (uint32_t)(rr >> 3) * 128 +
                      (uint32_t)(rr & 7) * 16;
            } else {
                const int R = i * a.NT + rr;
                off = slab * (size_t)(brows * kSlabK * 2) + (uint32_t)(g & 1) * (uint32_t)(brows * 16) +
                      (uint32_t)(R >> 3) * 128 + (uint32_t)(R & 7) * 16;
            }
            *reinterpret_cast<uint4*>(base + off) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    };
    // pass 2: digits of the cached groups, then of the rest (loaded again)
#pragma unroll
    for (int gi = 0; gi < kSplitCache; ++gi) {
        const int g = warp + gi * W;
        if (g < ngroups) emit(g, xc[gi]);
    }
    for (int g = warp + kSplitCache * W; g < ngroups; g += W) {
        unsigned long long xb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) xb[j] = load(8 * g + j);
        emit(g, xb);
    }
}

// ------------------------------------------------------------------ tensor-core GEMM

// v 2^E as a double from integer operations only (no FP64 instruction on the common path):
// the leading 53 bits of |v| (truncated). Results outside the normal range take the slow path.
__device__ __forceinline__ double ldexp_int(long long v, int E) {
    if (v == 0) return 0.0;
    const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
    const unsigned long long u = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)u);
    const int be = 1023 + 63 - lz + E;  // biased exponent of the result
    if (be <= 0 || be >= 2047) return scalbn((double)v, E);
    const unsigned long long m = (u << lz) >> 11;  // leading one at bit 52
    return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (m & 0x000FFFFFFFFFFFFFull)));
}

template <class T, int NT>
__global__ void __launch_bounds__(kGemmThreads, 2) tc_gemm_kernel(TcArgs<T> a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int cmul = (sizeof(T) == sizeof(cplx)) ? 2 : 1;
    const int S = a.S, nst = a.nst;
    const int nq = a.nprod;
    const int z = a.combine ? 0 : blockIdx.z;
    const int M = dimv(a.M[z], a.chi), N = dimv(a.N[z], a.chi), N2 = cmul * N;
    const int mt = blockIdx.y, nt = blockIdx.x;
    if (mt * kTileM >= M || nt * NT >= N2) return;

    const uint32_t slabA = (uint32_t)S * kSlabBytesA;        // all digits of one A slab
    const uint32_t slabB = (uint32_t)S * NT * kSlabK * 2;    // the stacked digits of one B slab
    const uint32_t stage_bytes = kStageSlabs * (slabA + slabB);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)nst * stage_bytes);  // full[nst], empty[nst], done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * nst + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* consumed = abort_flag + 1;
    int* s_expoB = const_cast<int*>(consumed) + 2;  // [nacc][NT] column scales of this tile
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nacc = a.combine ? nq : 1;  // accumulator sets (products) in this CTA
    for (int i = tid; i < nacc * NT; i += kGemmThreads) {
        const int q = a.combine ? i / NT : z;
        s_expoB[i] = a.expoB[(size_t)q * a.ntiles * NT + nt * NT + i % NT];
    }

    if (tid == 0) {
        for (int s = 0; s < 2 * nst + 1; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *abort_flag = 0;
        *consumed = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = *tmem_slot;

    // chunk c covers slabs [2 kc, 2 kc + 2) of accumulator set s; the sets follow each other
    int kslq[2] = {0, 0}, nch[2] = {0, 0};
    int total = 0;
    for (int s = 0; s < nacc; ++s) {
        const int q = a.combine ? s : z;
        kslq[s] = (cmul * dimv(a.K[q], a.chi) + kSlabK - 1) / kSlabK;
        nch[s] = (kslq[s] + kStageSlabs - 1) / kStageSlabs;
        total += nch[s];
    }
    const uint32_t bar_full = smem_u32(&bars[0]), bar_empty = smem_u32(&bars[nst]),
                   bar_done = smem_u32(&bars[2 * nst]);
    int issued = 0;

    if (warp == 0 && lane == 0) {  // producer: one bulk copy per operand per stage
        for (int c = 0; c < total; ++c) {
            const int st = c % nst, use = c / nst;
            if (use > 0 && !mbar_wait(bar_empty + 8 * st, (use - 1) & 1, a.wait_polls)) {
                *abort_flag = 1;
                break;
            }
            if (*abort_flag) break;
            const int s = c < nch[0] ? 0 : 1;
            const int kc = c - (s ? nch[0] : 0);
            const int q = a.combine ? s : z;
            const int nsl = min(kStageSlabs, kslq[s] - kStageSlabs * kc);
            const uint32_t fb = bar_full + 8 * st;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                         "r"((uint32_t)nsl * (slabA + slabB))
                         : "memory");
            const unsigned char* ga = a.planesA + (((size_t)q * a.mtiles + mt) * a.ksl + kStageSlabs * kc) * slabA;
            const unsigned char* gb = a.planesB + (((size_t)q * a.ntiles + nt) * a.ksl + kStageSlabs * kc) * slabB;
            unsigned char* sA = smem + (size_t)st * stage_bytes;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(sA)),
                "l"(ga), "r"((uint32_t)nsl * slabA), "r"(fb)
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(sA + kStageSlabs * slabA)),
                "l"(gb), "r"((uint32_t)nsl * slabB), "r"(fb)
                : "memory");
            issued = c + 1;
        }
    } else if (warp == 1 && lane == 0) {  // MMA issue: digit i of A against digits 0..S-1-i of B
        const uint64_t dA0 = sdesc(smem_u32(smem), kTileM * 16, 128);
        const uint64_t dB0 = sdesc(smem_u32(smem + kStageSlabs * slabA), (uint32_t)S * NT * 16, 128);
        int c = 0;
        for (; c < total; ++c) {
            const int st = c % nst, use = c / nst;
            if (*abort_flag) break;
            if (!mbar_wait(bar_full + 8 * st, use & 1, a.wait_polls)) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int s = c < nch[0] ? 0 : 1;
            const int kc = c - (s ? nch[0] : 0);
            const int nsl = min(kStageSlabs, kslq[s] - kStageSlabs * kc);
            const uint64_t stoff = (uint64_t)(st * stage_bytes) >> 4;  // descriptor start field, 16-byte units
            for (int ks = 0; ks < nsl; ++ks) {
                const uint64_t db = dB0 + stoff + ((uint64_t)(ks * slabB) >> 4);
                for (int i = 0; i < S; ++i) {
                    const uint64_t da = dA0 + stoff + ((uint64_t)(ks * slabA + i * kSlabBytesA) >> 4);
                    const uint32_t acc = (kc == 0 && ks == 0 && i == 0) ? 0u : 1u;  // i = 0 opens every order
                    // B digits 0..S-1-i are stacked along N: (S - i) NT rows, cut into MMAs of N <= 256
                    // (row r of the stack starts 16 r bytes into each K half of the slab)
                    const int ntot = (S - i) * NT;
                    for (int off = 0; off < ntot; off += 256) {
                        const int nn = min(256, ntot - off);
                        const uint32_t dt = tbase + (uint32_t)((s * S + i) * NT + off);
                        const uint32_t idesc = idesc_bf16(kTileM, nn);
                        const uint64_t dbo = db + (uint64_t)off;  // off rows x 16 bytes, in 16-byte units
                        asm volatile(
                            "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
                            "l"(da), "l"(dbo), "r"(idesc), "r"(acc));
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                bar_empty + 8 * st));
        }
        *consumed = c;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_done));
        if (a.tc_flops && c == total) {
            int slabs = 0;
            for (int s = 0; s < nacc; ++s) slabs += kslq[s];
            atomicAdd(a.tc_flops, 2.0 * kTileM * NT * kSlabK * (double)slabs * (S * (S + 1) / 2));
        }
    }
    __syncwarp();
    const bool done_ok = mbar_wait(bar_done, 0);
    __syncthreads();
    const bool ok = done_ok && !*abort_flag;
    if (!ok) {
        if (tid == 0) {
            atomicOr(a.err, DEVERR_TIMEOUT);
            // copies issued but never consumed: wait for them (bounded) before the CTA leaves
            for (int c = *consumed; c < issued; ++c) mbar_wait(bar_full + 8 * (c % nst), (c / nst) & 1);
        }
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and half w / 4 of the NT columns
        const int quarter = warp & 3, half = warp >> 2;
        const int row = mt * kTileM + quarter * 32 + lane;
        const bool rlive = row < M;
        int er[2] = {0, 0};
        for (int s = 0; s < nacc; ++s) {
            const int q = a.combine ? s : z;
            er[s] = a.expoA[(size_t)q * a.mtiles * kTileM + (rlive ? row : 0)];
        }
        const int b = a.bits;
        const int Ebase = -b * (S + 1);
        const int sh_hi = b * (S - 3);  // weight of the high half when S > 6
        unsigned long long mk = 0;
        T* C = a.C[z];
        constexpr int kHalf = NT / 2;
        for (int c8 = half * kHalf; c8 < (half + 1) * kHalf; c8 += 8) {
            double val[2][8];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (s >= nacc) break;
                // the S orders of 8 columns, loaded together: X = sum_t acc_t 2^(b (S-1-t))
                uint32_t v[kTcMaxDigits][8];
#pragma unroll
                for (int t = 0; t < kTcMaxDigits; ++t) {
                    if (t >= S) break;
                    const uint32_t addr =
                        tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((s * S + t) * NT + c8);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                        : "=r"(v[t][0]), "=r"(v[t][1]), "=r"(v[t][2]), "=r"(v[t][3]), "=r"(v[t][4]), "=r"(v[t][5]),
                          "=r"(v[t][6]), "=r"(v[t][7])
                        : "r"(addr));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                long long hi[8], lo[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) hi[j] = lo[j] = 0;
#pragma unroll
                for (int t = 0; t < kTcMaxDigits; ++t) {
                    if (t >= S) break;
                    const bool to_hi = S <= 6 || t < 3;  // one int64 holds X for S <= 6 (|X| < 2^60)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const long long iv = __float2int_rn(__uint_as_float(v[t][j]));
                        if (to_hi) hi[j] = (long long)((unsigned long long)hi[j] << b) + iv;
                        else lo[j] = (long long)((unsigned long long)lo[j] << b) + iv;
                    }
                }
                const int* eB = s_expoB + s * NT + c8;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int ec = eB[j];
                    double x;
                    if (er[s] >= kExpNonFinite || ec >= kExpNonFinite) x = __longlong_as_double(0x7FF8000000000000ll);
                    else if (S <= 6) x = ldexp_int(hi[j], er[s] + ec + Ebase);
                    else x = ldexp_int(hi[j], er[s] + ec + Ebase + sh_hi) + ldexp_int(lo[j], er[s] + ec + Ebase);
                    val[s][j] = x;
                }
            }
            if (!rlive) continue;
#pragma unroll
            for (int j = 0; j < 8; j += cmul) {
                const int col = (nt * NT + c8 + j) / cmul;
                if (col >= N) continue;
                T v0, v1;
                if constexpr (cmul == 2) {
                    v0 = mkc(val[0][j], val[0][j + 1]);
                    v1 = nacc > 1 ? mkc(val[1][j], val[1][j + 1]) : s_zero(T());
                } else {
                    v0 = val[0][j];
                    v1 = nacc > 1 ? val[1][j] : 0.0;
                }
                const T v = a.combine ? apply_f(a.op, v0, v1) : v0;
                C[(size_t)row * N + col] = v;
                const unsigned long long k = key_of(v);
                mk = k > mk ? k : mk;
            }
        }
        if (a.smax) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, mk, off);
                mk = o > mk ? o : mk;
            }
            if (lane == 0) {
                const double mag = key_to_mag(__longlong_as_double((long long)mk), T());
                atomicMax(a.smax, (unsigned long long)__double_as_longlong(mag));
            }
        }
        if (a.flops && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
            const double per = cmul == 2 ? 8.0 : 2.0;
            double f = 0.0;
            for (int s = 0; s < nacc; ++s) {
                const int q = a.combine ? s : z;
                f += per * (double)M * (double)N * (double)dimv(a.K[q], a.chi);
            }
            atomicAdd(a.flops, f);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(a.tmem_cols));
}

template <class T, int NT> cudaError_t set_attrs(size_t smem) {
    static std::mutex mu;
    static size_t done = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (smem <= done) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(tc_gemm_kernel<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done = smem;
    return e;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

int tc_nt_override() {
    static const int v = [] {
        const char* e = std::getenv("ACI_TC_NT");
        return e ? std::atoi(e) : 0;
    }();
    return v;
}

TcPlan tc_plan(int digits, bool cplx_values, int Mmax, int Nmax, int Kmax, int nprod, int combine, int nt_pref) {
    TcPlan p;
    const int cmul = cplx_values ? 2 : 1;
    p.S = digits;
    p.nacc = combine ? nprod : 1;
    // TMEM holds nacc * S * NT columns (<= 512). NT = 64 halves the re-reads of A's digit planes
    // (every N tile reads them again), but above 4 digits its tensor memory no longer fits two
    // CTAs per SM, and losing the overlap of one CTA's epilogue with the other's copies and MMAs
    // costs more (2048 x 2048 x 256 complex: bf16x6 0.43 vs 0.40 ms, bf16x8 0.53 vs 0.46 ms).
    // The S stacked B digits of an MMA are cut into MMAs of N <= 256. ACI_TC_NT overrides the
    // width where tensor memory allows it (tuning only).
    p.NT = (digits <= 4) ? 64 : 32;
    const int nt_want = nt_pref ? nt_pref : tc_nt_override();  // the contraction tuner's choice, else the override
    if ((nt_want == 32 || nt_want == 64) && (size_t)p.nacc * digits * nt_want <= 512) p.NT = nt_want;
    const long long K2 = (long long)cmul * std::max(Kmax, 1);
    p.bits = 7;
    while (p.bits > 2 && (long long)digits * K2 * ((1ll << p.bits) - 1) * ((1ll << p.bits) - 1) >= (1ll << 24))
        --p.bits;
    p.ksl = (int)((K2 + kSlabK - 1) / kSlabK);
    p.mtiles = (std::max(Mmax, 1) + kTileM - 1) / kTileM;
    p.ntiles = (int)(((long long)cmul * std::max(Nmax, 1) + p.NT - 1) / p.NT);
    const size_t slabB = (size_t)p.NT * kSlabK * 2;
    const size_t np = (size_t)std::max(nprod, 1);
    p.bytesA = align256(np * digits * p.mtiles * p.ksl * kSlabBytesA);
    p.bytesB = align256(np * digits * p.ntiles * p.ksl * slabB);
    p.bytesE = align256(sizeof(int) * np * ((size_t)p.mtiles * kTileM + (size_t)p.ntiles * p.NT));
    const size_t stage = (size_t)std::max(digits, 1) * kStageSlabs * (kSlabBytesA + slabB);  // A and B slabs
    uint32_t cols = 32;
    while (cols < (uint32_t)(p.nacc * digits * p.NT)) cols <<= 1;
    p.tmem_cols = cols;
    const size_t extra = 8 * (2 * 8 + 1) + 16 + sizeof(int) * 2 * 64;  // barriers, flags, column scales
    if (cols <= 256) {
        // two CTAs per SM (their tensor memory fits side by side): one's epilogue overlaps the
        // other's copies and MMAs; registers (<= 128 per thread) allow no third
        p.nst = (int)std::min<size_t>(4, (100 * 1024 - extra) / stage);
        p.smem = (size_t)p.nst * stage + extra;
    } else {
        // one CTA per SM: the shared-memory request keeps a second CTA (and its allocation) away
        p.nst = (int)std::min<size_t>(8, (200 * 1024 - extra) / stage);
        p.smem = std::max<size_t>((size_t)p.nst * stage + extra, 120 * 1024);
    }
    p.ok = digits >= kTcMinDigits && digits <= kTcMaxDigits && p.nst >= 1 && cols <= 512 && p.bits >= 3;
    return p;
}

size_t tc_scratch_bytes(const TcPlan& p) { return p.bytesA + p.bytesB + p.bytesE; }

template <class T>
cudaError_t launch_gemm_tc(const GemmArgs<T>& g, int Mmax, int Nmax, int Kmax, int digits, void* scratch,
                           size_t scratch_bytes, int* err, double* tc_flops, cudaStream_t st, long long wait_polls,
                           int nt_pref) {
    if (Mmax <= 0 || Nmax <= 0) return cudaSuccess;
    const bool cv = sizeof(T) == sizeof(cplx);
    const TcPlan p = tc_plan(digits, cv, Mmax, Nmax, Kmax, g.nprod, g.combine, nt_pref);
    if (!p.ok || tc_scratch_bytes(p) > scratch_bytes) return cudaErrorInvalidValue;
    TcArgs<T> a;
    for (int q = 0; q < 2; ++q) {
        a.A[q] = g.A[q];
        a.B[q] = g.B[q];
        a.C[q] = g.C[q];
        a.M[q] = g.M[q];
        a.N[q] = g.N[q];
        a.K[q] = g.K[q];
        a.lda[q] = g.lda[q];
        a.ldb[q] = g.ldb[q];
    }
    a.arow = g.arow;
    a.bcol = g.bcol;
    a.chi = g.chi;
    a.nprod = g.nprod;
    a.combine = g.combine;
    a.op = g.op;
    a.smax = g.smax;
    a.flops = g.flops;
    a.tc_flops = tc_flops;
    a.err = err;
    a.S = p.S;
    a.bits = p.bits;
    a.NT = p.NT;
    a.ksl = p.ksl;
    a.mtiles = p.mtiles;
    a.ntiles = p.ntiles;
    a.nst = p.nst;
    a.tmem_cols = p.tmem_cols;
    a.wait_polls = wait_polls;
    unsigned char* base = static_cast<unsigned char*>(scratch);
    a.planesA = base;
    a.planesB = base + p.bytesA;
    a.expoA = reinterpret_cast<int*>(base + p.bytesA + p.bytesB);
    a.expoB = a.expoA + (size_t)g.nprod * p.mtiles * kTileM;

    const int rows_cap = std::max(p.mtiles * kTileM, p.ntiles * p.NT);
    const int split_warps = std::min(kSplitMaxWarps, std::max(1, (2 * p.ksl + kSplitCache - 1) / kSplitCache));
    tc_split_kernel<T><<<dim3((rows_cap + 31) / 32, 2 * g.nprod), 32 * split_warps, 0, st>>>(a);
    const dim3 grid(p.ntiles, p.mtiles, g.combine ? 1 : g.nprod);
    cudaError_t e;
    if (p.NT == 32) {
        if ((e = set_attrs<T, 32>(p.smem)) != cudaSuccess) return e;
        tc_gemm_kernel<T, 32><<<grid, kGemmThreads, p.smem, st>>>(a);
    } else {
        if ((e = set_attrs<T, 64>(p.smem)) != cudaSuccess) return e;
        tc_gemm_kernel<T, 64><<<grid, kGemmThreads, p.smem, st>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t launch_gemm_tc<double>(const GemmArgs<double>&, int, int, int, int, void*, size_t, int*, double*,
                                            cudaStream_t, long long, int);
template cudaError_t launch_gemm_tc<cplx>(const GemmArgs<cplx>&, int, int, int, int, void*, size_t, int*, double*,
                                          cudaStream_t, long long, int);

}  // namespace aci
