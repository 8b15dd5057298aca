// Internal interfaces between the ACI driver (aci_api.cu) and its kernels.
#pragma once

#include "aci_common.cuh"

namespace aci {

// C = gather_rows(A) * gather_cols(B) (batch: one output per product) or
// C[0] = f(A^0 B^0, A^1 B^1) (combine). Row-major everything; ldc = N.
template <class T> struct GemmArgs {
    const T* A[kMaxInputs];
    const T* B[kMaxInputs];
    T* C[kMaxInputs];
    DimE M[kMaxInputs], N[kMaxInputs];
    DimE K[kMaxInputs], lda[kMaxInputs], ldb[kMaxInputs];
    const int* arow;  // optional row gather of A (shared by the products)
    const int* bcol;  // optional column gather of B
    const int* chi;   // device rank array the DimE refer to
    int nprod;
    int combine;
    OpParams<T> op;
    unsigned long long* smax;  // optional running max |C| (bits of a non-negative double)
    double* flops;             // optional: algorithmic flops of the launch are added here
    T* part;                   // scratch for partial tiles: gemm_part_elems(...) elements
    int* tile_count;           // zeroed counters: gemm_tile_counters(...) of them (left zeroed)
    int target_units;          // gemm_target_units(num_sms)
    int num_sms;
};

template <class T> void launch_gemm(const GemmArgs<T>& g, int Mmax, int Nmax, cudaStream_t st);
// Split-K granularity: about per_sm work units per SM (default kGemmUnitsPerSm; the contraction
// tuner of aci_opts.autotune chooses among 1, 2, 4 and 8 per shape class).
constexpr int kGemmUnitsPerSm = 4;
constexpr int kGemmMaxUnitsPerSm = 8;
int gemm_target_units(int num_sms, int per_sm = kGemmUnitsPerSm);
size_t gemm_part_elems(int Mmax, int Nmax, int nprod, int combine, int num_sms);
size_t gemm_tile_counters(int Mmax, int Nmax, int nprod);

// Tensor-core form of the same contractions (exact BF16 digit planes, FP32 accumulation in tensor
// memory): the operands and results of GemmArgs plus the digit-plane scratch.
constexpr int kTcMinDigits = 2;
constexpr int kTcMaxDigits = 8;

template <class T> struct TcArgs {
    const T* A[2];
    const T* B[2];
    T* C[2];
    DimE M[2], N[2], K[2], lda[2], ldb[2];
    const int* arow;
    const int* bcol;
    const int* chi;
    int nprod, combine;
    OpParams<T> op;
    unsigned long long* smax;
    double* flops;     // FP64-equivalent algorithmic flops (as gemm_kernel)
    double* tc_flops;  // optional: BF16 tensor-core flops issued
    int* err;
    int S, bits, NT, ksl, mtiles, ntiles, nst;
    uint32_t tmem_cols;
    unsigned char* planesA;  // [nprod][S][mtiles][ksl] slabs of 128 x 16 BF16
    unsigned char* planesB;  // [nprod][S][ntiles][ksl] slabs of NT x 16 BF16
    int* expoA;              // [nprod][mtiles * 128] row scale exponents
    int* expoB;              // [nprod][ntiles * NT] column scale exponents
    long long wait_polls;    // > 0: pipeline waits give up after that many polls (diagnostics); 0: 2 s
};

struct TcPlan {
    int S, bits, NT, nacc, ksl, mtiles, ntiles, nst;
    uint32_t tmem_cols;
    size_t bytesA, bytesB, bytesE, smem;
    bool ok;
};
// Kmax: largest K of the launch's products (complex counts once; the plan doubles it).
// nt_pref: the output tile width to use (32 or 64) where tensor memory allows it; 0 = the default rule.
TcPlan tc_plan(int digits, bool cplx_values, int Mmax, int Nmax, int Kmax, int nprod, int combine, int nt_pref = 0);
size_t tc_scratch_bytes(const TcPlan& p);
template <class T>
cudaError_t launch_gemm_tc(const GemmArgs<T>& g, int Mmax, int Nmax, int Kmax, int digits, void* scratch,
                           size_t scratch_bytes, int* err, double* tc_flops, cudaStream_t st,
                           long long wait_polls = 0, int nt_pref = 0);

template <class T> struct PrrluArgs {
    const T* Min;       // m x n row-major input, not modified
    DimE m, n;          // live shape (device-resolved)
    const int* chi;
    int chimax;         // rank cap
    int out_chi_idx;    // chi[out_chi_idx] = k on exit (-1: not written)
    int* k_out;         // optional device int
    double* eps_out;    // device double
    double* flops;      // optional: algorithmic flops of the factorisation are added here
    int* piv_rows;      // [kcap]
    int* piv_cols;      // [kcap]
    T* D;               // [kcap]
    T* L;               // optional, column-major m x kcap, leading dimension Lld
    int Lld;
    T* U;               // optional, row-major kcap x n, leading dimension Uld
    int Uld;
    double tol;         // tau = tol * S (rel) or tol (abs)
    int rel;
    const unsigned long long* smax;  // S for rel
    T* W;               // global working copy (column-major, ld mmax) when the block does not fit in shared memory
    unsigned long long* ll;  // exchange words: prrlu_ll_words(mmax, G, complex) of them
    unsigned int tagbase;    // tags are tagbase + step + 1; distinct per launch since the area was cleared
    int mmax, nmax;     // capacities of this launch
    int* err;           // device error flags (DevErr)
    int rook;           // 1: rook search (W holds prrlu_rook_scratch_elems, ll prrlu_rook_ll_words(G); L, U required)
    int no_coop;        // 1: no cooperative grid launch (the single-cluster kernel at every size)
    long long spin_limit;  // > 0: exchange waits give up after that many polls (diagnostics); 0: kSpinLimit
    // filled by launch_prrlu
    int epc, wcap_elems, wcap_cols;
    int grid_c;         // column groups of the 2D register variant (its cluster is grid_r x grid_c CTAs)
    int c2d_mbx;        // 1: the 2D variant exchanges candidates through mbarriers, not the cluster barrier
    // Live-shape split between the single-CTA variant and the variant chosen for the capacity:
    // a block with m <= small_m, n <= small_n and m n <= small_elems is factorised by the single-CTA
    // kernel and any other by the capacity's variant; each kernel returns at once when the block
    // is not its own (small_elems = 0: no single-CTA launch).
    int small_m, small_n, small_elems;
};

// Target entries of the pivot block per CTA: small blocks run in one CTA (no grid sync).
constexpr int kPrrluEpc = 2048;
// Steps per launch are < 2^13; tag bases are (launch number within a cleared area) << 13.
constexpr int kPrrluStepBits = 13;
constexpr unsigned int kPrrluMaxLaunches = (1u << (32 - kPrrluStepBits)) - 1;

template <class T> cudaError_t launch_prrlu(const PrrluArgs<T>& a, int G, cudaStream_t st);
int prrlu_grid(int mmax, int nmax, int num_sms);
int prrlu_rook_grid(int mmax, int nmax, int num_sms);
size_t prrlu_rook_ll_words(int G);
size_t prrlu_rook_scratch_elems(int mmax, int nmax, bool cplx_values);
size_t prrlu_ll_words(int mmax, int G, bool cplx_values);
// y[i] = 1 / x[i] with the reciprocal the pivot search uses (step-level entry point).
void launch_recip(const double* x, int n, double* y, cudaStream_t st);

// The pivot-proposer network (aci_mlp.cu): F <= kMlpMaxInputs inputs, two hidden layers of
// kMlpHidden units, one logit; parameters flat FP32 (W1, b1, W2, b2, W3, b3).
constexpr int kMlpHidden = 128;
constexpr int kMlpMaxInputs = 16;
size_t mlp_param_count(int F);
size_t mlp_train_scratch(int n);  // floats of scratch for launch_mlp_grad
void launch_mlp_forward(int n, int F, const float* X, const float* P, int fp16, float* z, float* a1, float* a2,
                        cudaStream_t st);
void launch_mlp_grad(int n, int F, const float* X, const float* y, float pos_weight, const float* P, float* G,
                     double* loss, float* scratch, cudaStream_t st);
void launch_mlp_adam(int count, float* p, const float* g, float* m, float* v, int t, float lr, float b1, float b2,
                     float eps, cudaStream_t st);

// The learned proposer's device side (aci_proposer.cu).
constexpr int kPropFeatures = 7;
template <class T> struct ProposerArgs {
    const T* A[2];        // Pi-A operands (rows = Pi rows), as the Pi block reads them
    const T* B[2];        // Pi-B operands (columns = Pi columns)
    DimE M, N, K[2], lda[2], ldb[2];
    const int* chi;
    int nprod;
    int d_row, d_col;     // local dimensions of the bond's two sites
    DimE chi_row, chi_col;  // chi_b (row parents), chi_{b+2} (column children)
    const int* prev_rows;   // the bond's pivots of the previous sweep, kprev of them
    const int* prev_cols;
    DimE kprev;
    float bond_frac;
    float* X;             // (mcap + ncap) x kPropFeatures
    int mcap, ncap;
    int* side_max;        // [4] order-preserving int images of the side maxima of features 0, 1
                          // (rows q = 0, 1, then columns); INT_MIN between calls
};
template <class T> void launch_features(const ProposerArgs<T>& a, cudaStream_t st);
struct TopkArgs {
    const float* z;       // (mcap + ncap) scores
    DimE M, N, kprev;
    const int* chi;
    int mcap, ncap;
    float keep;
    int* sel_rows;        // [mcap] kept row indices, ascending
    int* sel_cols;        // [ncap]
    int slot_rows, slot_cols;  // chi[slot] <- the kept counts
};
size_t topk_smem(int mcap, int ncap);
cudaError_t launch_topk(const TopkArgs& t, cudaStream_t st);
void launch_map_pivots(const int* chi, int kslot, int* prow, int* pcol, const int* sel_rows, const int* sel_cols,
                       cudaStream_t st);
struct RecordArgs {
    const float* X;
    DimE M, N, k;
    const int* chi;
    int mcap;
    const int* prow;
    const int* pcol;
    float* buf;                 // records of kPropFeatures + 1 floats
    long long capacity;         // records
    unsigned long long* count;  // device counter (records requested so far)
};
void launch_record(const RecordArgs& r, cudaStream_t st);

// Per-bond buffers used by the output assembly.
template <class T> struct BondBuf {
    const T* Pi;   // m_b x n_b row-major
    const int* prow;
    const int* pcol;
    const T* D;
    const T* Lm;   // column-major m_b x kcap, ld Lld
    const T* Um;   // row-major kcap x n_b, ld Uld
    int Lld, Uld;
};

// Y_s = T_s P_s^-1 for every site s (CI-canonical output), into Y[s] (row-major, contiguous).
template <class T> struct AssembleArgs {
    int L;
    const int* chi;   // device ranks
    const int* d;     // device local dimensions
    const BondBuf<T>* bonds;  // [L-1] device array
    T* const* Y;      // [L] device array of output pointers
};
// Rmax: the largest rows chi_s d_s of a site, Kmax: the largest rank chi_{s+1} (capacities).
template <class T> void launch_assemble(const AssembleArgs<T>& a, int Rmax, int Kmax, cudaStream_t st);

// Y = T P^-1 with dense LI, D, UJ (k x k row-major): step-level entry point.
template <class T> void launch_apply_pinv(const T* Tm, int R, int k, const T* LI, const T* D,
                                          const T* UJ, T* Y, cudaStream_t st);

// SplitMix64 counter-based random cores: entry e of the concatenation (site offsets off[s]).
template <class T> void launch_tt_random(uint64_t seed, int L, const long long* off_host,
                                         const long long* count_host, T* const* cores_host,
                                         cudaStream_t st);

// End-of-iteration bookkeeping on the device (one CTA): rank growth, fixed point, max eps.
struct IterFlags {
    int grew;
    int fixed;
    int err;
    int pad;
    double emax;
    double S;
};
// Gathers of the overlapped sweep: dst[r * dld + c] = src[gather_row(r) * sld + gather_col(c)]
// for r < rows, c < cols (shapes read on the device), up to 1 + kMaxInputs independent jobs per launch.
// One job may also fold max |dst| into *smax (bits of a non-negative double, as the contractions).
template <class T> struct GatherJob {
    const T* src;
    T* dst;
    DimE rows, cols, sld, dld;
    const int* ridx;  // see gather_row
    int rblk;
    const int* cidx;  // see gather_col
    DimE cblk, cstride;
};
constexpr int kGatherJobs = 1 + kMaxInputs;
template <class T> struct GatherArgs {
    GatherJob<T> job[kGatherJobs];
    int njobs;
    int smax_job;  // job whose values feed smax, -1 for none
    const int* chi;
    unsigned long long* smax;
};
template <class T> void launch_gather(const GatherArgs<T>& a, long long max_elems, int num_sms, cudaStream_t st);
// 1: pivot searches and gathers are launched with programmatic dependent launch (ACI_PDL=0: off).
int prrlu_pdl_mode();

// Pivot history of a call (aci_stats.hist_*): copies chi[kidx] pivots of one local update.
struct HistArgs {
    const int* chi;
    int kidx;
    const int* prow;
    const int* pcol;
    int b, nb, kstride, nslots;
    int slot;         // >= 0: this slot; < 0: 1 + 2 (*iter - 1) + half
    int half;
    const int* iter;  // device iteration counter
    int* rank;        // [nslots][nb]
    int* rows;        // [nslots][nb][kstride]
    int* cols;
};
void launch_hist(const HistArgs& h, cudaStream_t st);
void launch_hist_tick(int* iter, cudaStream_t st);

// dst[e] = (double)src[e] for e < n (FP32 / complex64 inputs widened on load).
void launch_promote(const float* src, long long n, double* dst, cudaStream_t st);

// FP64 multiply-add throughput probe: `blocks` CTAs of 512 threads, `iters` rounds of the chains.
double fp64_probe_flops(int blocks, int iters);
void launch_fp64_probe(const double* seed, int blocks, int iters, double* out, cudaStream_t st);

void launch_iter_check(int L, const int* chi, int* chi_prev, int* const* pcol, int* const* jprev,
                       const double* eps_lr, const double* eps_rl, const unsigned long long* smax,
                       const int* err, IterFlags* flags, int snapshot_only, cudaStream_t st);

}  // namespace aci
