// Host driver of the ACI sweep (Algorithm 1) and the C ABI declared in include/aci.h and
// include/aci_kernels.h. Every arithmetic step runs in the library's kernels; the host only
// lays out buffers, enqueues launches on the context stream, and reads one small flag
// record per sweep (the stop test of Algorithm 1).
//
// Data layout in HBM for one call (0-based sites s = 0..L-1, bond b joins sites b and b+1):
//   chi[0..L]      output ranks (device), chi[b+1] = |I_b| = |J_{b+1}|, set by bond b's pivots
//   LX[n][s]       L^n_{s-1} X^n_s, (chi[s] d_s) x r^n_{s+1} row-major; LX[n][0] aliases X^n_0
//   XR[n][s]       X^n_s R^n_{s+1}, r^n_s x (d_s chi[s+1]) row-major; XR[n][L-1] aliases X^n_{L-1}
//   Pi[b]          f(LX[.][b] XR[.][b+1]), (chi[b] d_b) x (d_{b+1} chi[b+2]) row-major
//   prow/pcol[b]   bond b's pivots (positions in Pi[b]); D[b], Lm[b] (col-major), Um[b] (row-major)
// The frames L^n_b = rows prow[b] of LX[n][b] and R^n_{s} = columns pcol[s-1] of XR[n][s] are
// never materialised: the next contraction gathers them on load. LX[.][b] from a left-to-right
// sweep is reused by the following right-to-left sweep at the same bond, and XR[.][b+1] from a
// right-to-left sweep by the next left-to-right sweep (their frames have not changed).
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include <map>
#include <chrono>
#include <thread>
#include <atomic>

#include "../../include/aci.h"
#include "../../include/aci_kernels.h"
#include "aci_internal.h"

using aci::cplx;
using aci::DimE;
using aci::dimc;
using aci::dimr;

struct aci_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    aci_alloc_fn alloc = nullptr;
    aci_free_fn free_fn = nullptr;
    void* user = nullptr;
    std::string err;
    int num_sms = 0;
    unsigned long long epoch = 1;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    aci::IterFlags* hflags = nullptr;  // pinned
    long long launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> evfree;  // reusable events for per-kernel timing
    std::vector<cudaEvent_t> evall;
    cudaStream_t side = nullptr;      // second stream of the overlapped sweep (created on first use)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool own_stream = false;          // a batch worker owns its stream
    bool no_coop = false;             // a batch worker: no cooperative grids (others run beside it)
    std::vector<aci_ctx*> workers;    // batch workers (own streams, scratch and graphs)
    std::vector<cudaEvent_t> worker_ev;
    cudaEvent_t evb = nullptr;
    // Concurrency autotuner of aci_elementwise_batch (batch_streams = 0): per batch-size class
    // (floor(log2 n)), the candidate stream counts are tried on successive calls, each timed on the
    // host around the whole call; afterwards the best rate is used.
    struct BatchTune {
        std::vector<int> cand;
        std::vector<double> rate;
        int best = 0;
    };
    std::map<int, BatchTune> batch_tune;
    // learned proposer (ACI_PIVOT_PROPOSED) and training-data recording
    const float* prop_params = nullptr;
    float prop_keep = 1.25f;
    float* rec_buf = nullptr;
    long long rec_cap = 0;
    unsigned long long* rec_count = nullptr;
    // diagnostic wait limits (aci_set_wait_limits); 0 = the defaults
    long long exchange_polls = 0;
    long long pipeline_polls = 0;
    // split-K granularity (FP64) and output tile width (digit planes) per contraction shape class,
    // from the tuner of aci_opts.autotune
    std::map<unsigned long long, int> gemm_units;
    std::map<unsigned long long, int> tc_widths;
};

namespace {

struct Fail {
    aci_status st;
};

// SMs the side stream's contractions leave to the pivot search running beside them (its largest
// cluster); ACI_SIDE_RESERVE overrides it (launch-shape tuning only: results do not change).
int side_reserve() {
    static const int v = [] {
        const char* e = std::getenv("ACI_SIDE_RESERVE");
        return e ? std::max(0, std::atoi(e)) : 16;
    }();
    return v;
}

void fail(aci_ctx* ctx, aci_status st, const std::string& msg) {
    ctx->err = msg;
    throw Fail{st};
}

void ck(aci_ctx* ctx, cudaError_t e, const char* what) {
    if (e != cudaSuccess) fail(ctx, ACI_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(aci_ctx* ctx, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (ctx->alloc) {
        p = ctx->alloc(bytes, ctx->user);
    } else {
        if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess) p = nullptr;
    }
    if (!p) fail(ctx, ACI_E_ALLOC, "device allocation of " + std::to_string(bytes) + " bytes failed");
    return p;
}

void dev_free(aci_ctx* ctx, void* p) {
    if (!p) return;
    if (ctx->free_fn) ctx->free_fn(p, ctx->user);
    else cudaFreeAsync(p, ctx->stream);
}

// Grow the context workspace to at least `bytes`.
char* workspace(aci_ctx* ctx, size_t bytes) {
    if (bytes > ctx->ws_bytes) {
        if (ctx->ws) dev_free(ctx, ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
        const size_t want = bytes + bytes / 8;
        ctx->ws = dev_alloc(ctx, want);
        ctx->ws_bytes = want;
    }
    return static_cast<char*>(ctx->ws);
}

// Bump allocator over the workspace; the same layout routine runs once to size, once to carve.
struct Carver {
    char* base = nullptr;
    size_t off = 0;
    template <class U> U* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        U* p = base ? reinterpret_cast<U*>(base + off) : nullptr;
        off += count * sizeof(U);
        return p;
    }
};

void note_launch(aci_ctx* ctx, const char* what) {
    ctx->launches++;
    ck(ctx, cudaGetLastError(), what);
}

bool valid_precision(int p) {
    return p == ACI_PREC_FP64 || (p >= aci::kTcMinDigits && p <= aci::kTcMaxDigits);
}

long long sat_mul(long long a, long long b, long long cap) {
    if (a >= cap || b >= cap) return cap;
    long long v = a * b;
    return v > cap ? cap : v;
}

template <class T>
aci::OpParams<T> make_op(const aci_op& op);
template <>
aci::OpParams<double> make_op<double>(const aci_op& op) {
    aci::OpParams<double> p;
    p.kind = op.kind;
    for (int i = 0; i < 4; ++i) p.c[i] = op.c[i][0];
    return p;
}
template <>
aci::OpParams<cplx> make_op<cplx>(const aci_op& op) {
    aci::OpParams<cplx> p;
    p.kind = op.kind;
    for (int i = 0; i < 4; ++i) p.c[i] = aci::mkc(op.c[i][0], op.c[i][1]);
    return p;
}

// ------------------------------------------------------------------------------------------
// One ACI call (Algorithm 1) for scalar type T.
template <class T>
struct Run {
    aci_ctx* ctx;
    cudaStream_t st;
    int L = 0, N = 0, chimax = 0, maxit = 20, rel = 1, prof = 0;
    int digits = 0;            // 0: FP64 contractions; 2..8: BF16 digit planes on the tensor cores
    int rook = 0;              // pivot search: 0 full, 1 rook
    int no_coop = 0;           // concurrent batch worker: pivot searches stay within one cluster
    int proposed = 0;          // ACI_PIVOT_PROPOSED: learned candidate restriction in left-to-right sweeps
    bool recording = false;    // append (features, pivot-or-not) of full left-to-right sweeps
    float* pfeat = nullptr;    // proposer features, (mcap + ncap) x kPropFeatures
    float* pscore = nullptr;   // proposer scores
    int* psel_rows = nullptr;
    int* psel_cols = nullptr;
    int* pside = nullptr;      // [4] side maxima of the proposer's norm features
    size_t pcand = 1;          // largest mcap + ncap
    int overlap_opt = ACI_OVERLAP_AUTO;
    int overlap = 0;           // overlapped schedule (aci_overlap) in effect
    T* Qb[aci::kMaxInputs] = {};    // half-products over all candidate rows / columns
    T* Pfull = nullptr;             // Pi over all candidate rows / columns
    size_t qcap = 1, pfcap = 1;
    // per-kernel-class accounting (aci_kernel_class)
    double kms[4] = {0, 0, 0, 0};
    long long kcount[4] = {0, 0, 0, 0};
    double* kflops = nullptr;  // device [4]: algorithmic flops, then [4] tensor-core flops
    struct Pend {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Pend> pend;

    cudaEvent_t get_event() {
        if (ctx->evfree.empty()) {
            cudaEvent_t e;
            ck(ctx, cudaEventCreate(&e), "cudaEventCreate");
            ctx->evall.push_back(e);
            return e;
        }
        cudaEvent_t e = ctx->evfree.back();
        ctx->evfree.pop_back();
        return e;
    }
    cudaEvent_t pre(int) {
        if (!prof) return nullptr;
        cudaEvent_t e = get_event();
        ck(ctx, cudaEventRecord(e, st), "event");
        return e;
    }
    void post(int cls, cudaEvent_t a, const char* what) {
        note_launch(ctx, what);
        kcount[cls]++;
        if (!prof) return;
        cudaEvent_t b = get_event();
        ck(ctx, cudaEventRecord(b, st), "event");
        pend.push_back({cls, a, b});
    }
    // After a stream sync: fold the finished event pairs into kms.
    // keep = true: the pairs belong to a captured graph and are read again after the next replay.
    void harvest(bool keep = false) {
        for (auto& q : pend) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) kms[q.cls] += ms;
            if (!keep) {
                ctx->evfree.push_back(q.a);
                ctx->evfree.push_back(q.b);
            }
        }
        if (!keep) pend.clear();
    }
    double* flops_of(int cls) { return prof ? kflops + cls : nullptr; }
    double tol = 0;
    uint64_t seed = 0;
    aci::OpParams<T> op;
    std::vector<int> d;                    // [L]
    std::vector<std::vector<int>> r;       // r[n][0..L] input ranks
    std::vector<int> cap, ry;              // [L+1]
    std::vector<int> mcap, ncap, kcap;     // per bond
    bool host_in = false;
    const aci_tt* in[aci::kMaxInputs] = {};
    const aci_tt* init = nullptr;

    // device buffers
    std::vector<const T*> Xv[aci::kMaxInputs];
    std::vector<T*> Xcopy[aci::kMaxInputs];
    std::vector<T*> LX[aci::kMaxInputs], XR[aci::kMaxInputs], Yinit, Ysc, Pi, D, Lm, Um;
    std::vector<int*> prow, pcol, jprev;
    T* Minit[2] = {nullptr, nullptr};
    int *chi = nullptr, *chi_prev = nullptr, *dd = nullptr, *err = nullptr;
    double *eps_lr = nullptr, *eps_rl = nullptr, *eps_junk = nullptr;
    unsigned long long *smax = nullptr, *initmax = nullptr;
    aci::IterFlags* flags = nullptr;
    T* ones = nullptr;
    T* W = nullptr;
    T* gpart = nullptr;                 // GEMM partial tiles
    int* gcount = nullptr;              // GEMM per-tile counters (kept zeroed)
    size_t gpart_elems = 1, gcount_n = 1;
    unsigned char* tcbuf = nullptr;     // digit planes and scales of the tensor-core contractions
    size_t tc_bytes = 0;
    unsigned long long* ll = nullptr;  // pivot-search exchange words
    size_t ll_words = 0;
    unsigned int prrlu_launches = 0;   // launches since the exchange area was last cleared
    int Gmax = 1;
    size_t wcap = 0;
    int mmax_all = 1;
    aci::BondBuf<T>* bonds_dev = nullptr;
    T** Yptr_dev = nullptr;
    int** pcol_dev = nullptr;
    int** jprev_dev = nullptr;

    // contraction tuner (aci_opts.autotune): the shape classes this call launches
    int autotune = 0;
    struct GemmShape {
        int M, N, K, nprod, combine;
    };
    std::vector<GemmShape> gemm_shapes;
    // pivot history of the call (aci_stats.hist_*): one slot per local update and bond
    bool hist_on = false;
    int hist_slots = 0;
    int *hist_rank = nullptr, *hist_rows = nullptr, *hist_cols = nullptr, *hist_iter = nullptr;

    static constexpr bool is_cplx = sizeof(T) == sizeof(cplx);

    const T* Xp(int n, int s) const { return Xv[n][s]; }

    // Tag base of the next pivot-search launch; clears the exchange area when the tags of
    // this area are used up (launches since the last clear < 2^19).
    unsigned int next_tagbase() {
        if (prrlu_launches >= aci::kPrrluMaxLaunches) {
            ck(ctx, cudaMemsetAsync(ll, 0, ll_words * sizeof(unsigned long long), st), "clear exchange");
            prrlu_launches = 0;
        }
        ++prrlu_launches;
        return prrlu_launches << aci::kPrrluStepBits;
    }

    void layout(Carver& c) {
        for (int n = 0; n < N; ++n) {
            Xcopy[n].assign(L, nullptr);
            if (host_in)
                for (int s = 0; s < L; ++s)
                    Xcopy[n][s] = c.take<T>((size_t)r[n][s] * d[s] * r[n][s + 1]);
            LX[n].assign(L, nullptr);
            XR[n].assign(L, nullptr);
            for (int s = 1; s < L; ++s) LX[n][s] = c.take<T>((size_t)cap[s] * d[s] * r[n][s + 1]);
            for (int s = 0; s + 1 < L; ++s) XR[n][s] = c.take<T>((size_t)r[n][s] * d[s] * cap[s + 1]);
        }
        const int nb = std::max(L - 1, 0);
        Pi.assign(nb, nullptr);
        D.assign(nb, nullptr);
        Lm.assign(nb, nullptr);
        Um.assign(nb, nullptr);
        prow.assign(nb, nullptr);
        pcol.assign(nb, nullptr);
        jprev.assign(nb, nullptr);
        for (int b = 0; b < nb; ++b) {
            Pi[b] = c.take<T>((size_t)mcap[b] * ncap[b]);
            D[b] = c.take<T>(kcap[b]);
            Lm[b] = c.take<T>((size_t)mcap[b] * kcap[b]);
            Um[b] = c.take<T>((size_t)kcap[b] * ncap[b]);
            prow[b] = c.take<int>(kcap[b]);
            pcol[b] = c.take<int>(kcap[b]);
            jprev[b] = c.take<int>(kcap[b]);
        }
        Yinit.assign(L, nullptr);
        Ysc.assign(L, nullptr);
        size_t minit = 1;
        for (int s = 0; s < L; ++s) {
            Yinit[s] = c.take<T>((size_t)ry[s] * d[s] * ry[s + 1]);
            Ysc[s] = c.take<T>((size_t)cap[s] * d[s] * cap[s + 1]);
            minit = std::max(minit, (size_t)ry[s] * d[s] * cap[s + 1]);
        }
        Minit[0] = c.take<T>(minit);
        Minit[1] = c.take<T>(minit);
        chi = c.take<int>(L + 3);  // ranks, then the proposer's kept row / column counts
        chi_prev = c.take<int>(L + 1);
        dd = c.take<int>(L);
        err = c.take<int>(1);
        eps_lr = c.take<double>(std::max(nb, 1));
        eps_rl = c.take<double>(std::max(nb, 1));
        eps_junk = c.take<double>(1);
        kflops = c.take<double>(8);
        smax = c.take<unsigned long long>(1);
        initmax = c.take<unsigned long long>(1);
        flags = c.take<aci::IterFlags>(1);
        ones = c.take<T>(1);
        W = c.take<T>(wcap);
        ll = c.take<unsigned long long>(ll_words);
        gpart = c.take<T>(gpart_elems);
        gcount = c.take<int>(gcount_n);
        tcbuf = c.take<unsigned char>(tc_bytes);
        bonds_dev = c.take<aci::BondBuf<T>>(std::max(nb, 1));
        if (proposed || recording) {
            pfeat = c.take<float>(pcand * aci::kPropFeatures);
            pscore = c.take<float>(pcand);
            psel_rows = c.take<int>(pcand);
            psel_cols = c.take<int>(pcand);
            pside = c.take<int>(4);
        }
        if (overlap) {
            for (int n = 0; n < N; ++n) Qb[n] = c.take<T>(qcap);
            Pfull = c.take<T>(pfcap);
        }
        if (hist_on) {
            hist_rank = c.take<int>((size_t)hist_slots * nb);
            hist_rows = c.take<int>((size_t)hist_slots * nb * chimax);
            hist_cols = c.take<int>((size_t)hist_slots * nb * chimax);
            hist_iter = c.take<int>(1);
        }
        Yptr_dev = c.take<T*>(L);
        pcol_dev = c.take<int*>(std::max(nb, 1));
        jprev_dev = c.take<int*>(std::max(nb, 1));
    }

    // exchange words and scratch of one pivot search of capacity m x n
    void size_pivot_search(int m, int n) {
        if (rook) {
            const int kc = std::min(std::min(m, n), chimax);
            if (kc > (is_cplx ? 2048 : 4096)) fail(ctx, ACI_E_SHAPE, "rook search supports at most 4096 (real) / 2048 (complex) pivots per bond");
            const int G = aci::prrlu_rook_grid(m, n, ctx->num_sms);
            Gmax = std::max(Gmax, G);
            ll_words = std::max(ll_words, aci::prrlu_rook_ll_words(G));
            wcap = std::max(wcap, aci::prrlu_rook_scratch_elems(m, n, is_cplx));
        } else {
            const int G = aci::prrlu_grid(m, n, ctx->num_sms);
            Gmax = std::max(Gmax, G);
            ll_words = std::max(ll_words, aci::prrlu_ll_words(m, G, is_cplx));
        }
    }

    void plan_sizes() {
        cap.assign(L + 1, 1);
        const long long big = 1LL << 40;
        for (int s = 1; s < L; ++s) {
            long long pl = 1, pr = 1;
            for (int t = 0; t < s; ++t) pl = sat_mul(pl, d[t], big);
            for (int t = s; t < L; ++t) pr = sat_mul(pr, d[t], big);
            cap[s] = (int)std::min<long long>({(long long)chimax, pl, pr});
        }
        ry.assign(L + 1, 1);
        for (int s = 1; s < L; ++s) {
            int v = cap[s];
            for (int n = 0; n < N; ++n) v = std::min(v, r[n][s]);
            if (init) {
                if (init->rank[s] > cap[s])
                    fail(ctx, ACI_E_SHAPE, "init rank exceeds min(max_rank, prod d left, prod d right)");
                v = (int)init->rank[s];
            }
            ry[s] = v;
        }
        const int nb = std::max(L - 1, 0);
        mcap.assign(nb, 0);
        ncap.assign(nb, 0);
        kcap.assign(nb, 0);
        wcap = 1;
        mmax_all = 1;
        Gmax = 1;
        for (int b = 0; b < nb; ++b) {
            mcap[b] = cap[b] * d[b];
            ncap[b] = d[b + 1] * cap[b + 2];
            kcap[b] = cap[b + 1];
            wcap = std::max(wcap, (size_t)mcap[b] * ncap[b]);
            mmax_all = std::max(mmax_all, mcap[b]);
            size_pivot_search(mcap[b], ncap[b]);
            pcand = std::max(pcand, (size_t)mcap[b] + ncap[b]);
            if ((long long)mcap[b] * ncap[b] >= (1LL << 31))
                fail(ctx, ACI_E_SHAPE, "a Pi block would exceed 2^31 entries");
        }
        int rmax = 1;
        for (int n = 0; n < N; ++n)
            for (int s = 0; s <= L; ++s) rmax = std::max(rmax, r[n][s]);
        for (int s = 0; s <= L; ++s) rmax = std::max(rmax, ry[s]);
        // optional: a contraction of the overlapped schedule, which falls back to the plain one
        gemm_shapes.clear();
        auto need = [&](int Mm, int Nm, int nprod, int combine, bool optional = false) {
            gemm_shapes.push_back({Mm, Nm, rmax, nprod, combine});
            if (digits) {  // K of every contraction is an input rank or an initial-guess rank
                const aci::TcPlan p = aci::tc_plan(digits, is_cplx, Mm, Nm, rmax, nprod, combine);
                for (int nt : {32, 64}) {  // the tuner may choose either width: room for both
                    const aci::TcPlan q = aci::tc_plan(digits, is_cplx, Mm, Nm, rmax, nprod, combine, nt);
                    if (q.ok) tc_bytes = std::max(tc_bytes, aci::tc_scratch_bytes(q));
                }
                if (!p.ok) {
                    if (optional) {
                        overlap = 0;
                        return;
                    }
                    fail(ctx, ACI_E_SHAPE, "contraction too large for the digit-plane precision");
                }
                tc_bytes = std::max(tc_bytes, aci::tc_scratch_bytes(p));
            }
            gpart_elems = std::max(gpart_elems, aci::gemm_part_elems(Mm, Nm, nprod, combine, ctx->num_sms));
            gcount_n = std::max(gcount_n, aci::gemm_tile_counters(Mm, Nm, nprod));
        };
        const int dmax = *std::max_element(d.begin(), d.end());
        overlap = 0;
        if (overlap_opt != ACI_OVERLAP_OFF && nb >= 2 && (overlap_opt == ACI_OVERLAP_ON || (dmax == 2 && !no_coop)))
            overlap = 1;
        if (overlap) {  // the contractions of side_lr / side_rl and their buffers
            qcap = pfcap = 1;
            const long long lim = 1LL << 31;
            for (int b = 1; b < nb; ++b) {
                const long long rows = (long long)mcap[b - 1] * d[b];
                need((int)std::min(rows, lim - 1), ncap[b], N, 1, true);
                pfcap = std::max<size_t>(pfcap, (size_t)rows * ncap[b]);
                for (int n = 0; n < N; ++n) qcap = std::max<size_t>(qcap, (size_t)rows * r[n][b + 1]);
                need(mcap[b - 1], d[b] * rmax, N, 0, true);
            }
            for (int b = 0; b + 1 < nb; ++b) {
                const long long cols = (long long)d[b + 1] * ncap[b + 1];
                need(mcap[b], (int)std::min(cols, lim - 1), N, 1, true);
                pfcap = std::max<size_t>(pfcap, (size_t)mcap[b] * cols);
                for (int n = 0; n < N; ++n) qcap = std::max<size_t>(qcap, (size_t)r[n][b + 1] * cols);
                need(rmax * d[b + 1], ncap[b + 1], N, 0, true);
            }
            if (pfcap >= (size_t)lim || qcap >= (size_t)lim) overlap = 0;
        }
        for (int b = 0; b < nb; ++b) need(mcap[b], ncap[b], N, 1);
        for (int s = 0; s < L; ++s) {
            need(cap[s], dmax * rmax, N, 0);           // left half-products
            need(rmax * dmax, cap[s + 1], N, 0);       // right half-products
            need(ry[s] * d[s], cap[s + 1], 1, 0);      // initial CI
        }
        need(dmax, 1, N, 1);                           // single site
        for (int s = 1; s < L; ++s) {
            const int m = ry[s], n = d[s] * cap[s + 1];
            wcap = std::max(wcap, (size_t)m * n);
            mmax_all = std::max(mmax_all, m);
            size_pivot_search(m, n);
        }
    }

    // ---------------------------------------------------------------- contraction tuner
    // Shape class: ceil(log2) of M, N and K (capacities), products, Pi (combine) or frame form, dtype.
    static int lg(int v) {
        int l = 0;
        while ((1 << l) < v && l < 30) ++l;
        return l;
    }
    static unsigned long long shape_key(int M, int N, int K, int nprod, int combine) {
        return ((unsigned long long)lg(M) << 24) | ((unsigned long long)lg(N) << 16) | ((unsigned long long)lg(K) << 8) |
               ((unsigned long long)nprod << 2) | ((unsigned long long)combine << 1) | (is_cplx ? 1ull : 0ull);
    }
    int tc_width(int M, int N, int K, int nprod, int combine) const {
        if (ctx->tc_widths.empty()) return 0;
        auto it = ctx->tc_widths.find(shape_key(M, N, K, nprod, combine) ^ ((unsigned long long)digits << 40));
        return it == ctx->tc_widths.end() ? 0 : it->second;
    }
    int units_per_sm(int M, int N, int K, int nprod, int combine) const {
        if (ctx->gemm_units.empty()) return aci::kGemmUnitsPerSm;
        auto it = ctx->gemm_units.find(shape_key(M, N, K, nprod, combine));
        return it == ctx->gemm_units.end() ? aci::kGemmUnitsPerSm : it->second;
    }
    // Time every candidate granularity on each untuned shape class of this call (operands of the
    // class's size, zero-filled: the FP64 pipe's timing does not depend on the values) and keep the
    // fastest. Runs on the context stream before the sweeps.
    void tune_contractions() {
        static const int cand[] = {1, 2, 4, 8};
        static const int widths[] = {32, 64};
        std::vector<GemmShape> todo;
        std::map<unsigned long long, int> seen;
        const unsigned long long dkey = (unsigned long long)digits << 40;
        for (const GemmShape& g : gemm_shapes) {
            const unsigned long long k = shape_key(g.M, g.N, g.K, g.nprod, g.combine) ^ dkey;
            if ((digits ? ctx->tc_widths.count(k) : ctx->gemm_units.count(k)) || seen.count(k)) continue;
            seen[k] = 1;
            todo.push_back(g);
        }
        if (todo.empty()) return;
        size_t ea = 1, eb = 1, ec = 1;
        for (const GemmShape& g : todo) {
            ea = std::max(ea, (size_t)g.M * g.K);
            eb = std::max(eb, (size_t)g.K * g.N);
            ec = std::max(ec, (size_t)g.M * g.N);
        }
        const size_t bytes = sizeof(T) * (ea + eb + 2 * ec) + 1024;
        char* buf = static_cast<char*>(dev_alloc(ctx, bytes));
        cudaEvent_t e0 = get_event(), e1 = get_event();
        try {
            ck(ctx, cudaMemsetAsync(buf, 0, bytes, st), "tuner operands");
            T* A = reinterpret_cast<T*>(buf);
            T* B = A + ea;
            T* C = B + eb;
            for (const GemmShape& sh : todo) {
                aci::GemmArgs<T> g = gemm_base();
                g.combine = sh.combine;
                g.nprod = sh.nprod;
                for (int n = 0; n < sh.nprod; ++n) {
                    g.A[n] = A;
                    g.B[n] = B;
                    g.C[n] = sh.combine ? C : C + (n & 1) * ec;
                    g.M[n] = dimc(sh.M);
                    g.N[n] = dimc(sh.N);
                    g.K[n] = dimc(sh.K);
                    g.lda[n] = dimc(sh.K);
                    g.ldb[n] = dimc(sh.N);
                }
                g.chi = chi;
                g.part = gpart;
                g.tile_count = gcount;
                g.num_sms = ctx->num_sms;
                int best = digits ? 0 : aci::kGemmUnitsPerSm;
                float best_ms = 1e30f;
                const int ncand = digits ? 2 : 4;
                for (int ci = 0; ci < ncand; ++ci) {
                    const int c = digits ? widths[ci] : cand[ci];
                    if (digits) {
                        const aci::TcPlan q = aci::tc_plan(digits, is_cplx, sh.M, sh.N, sh.K, sh.nprod, sh.combine, c);
                        if (!q.ok || q.NT != c || aci::tc_scratch_bytes(q) > tc_bytes) continue;
                    } else {
                        g.target_units = aci::gemm_target_units(ctx->num_sms, c);
                    }
                    auto launch = [&]() {
                        if (digits)
                            ck(ctx, aci::launch_gemm_tc<T>(g, sh.M, sh.N, sh.K, digits, tcbuf, tc_bytes, err, nullptr, st,
                                                           ctx->pipeline_polls, c),
                               "tuner");
                        else
                            aci::launch_gemm<T>(g, sh.M, sh.N, st);
                    };
                    launch();  // warm-up
                    ck(ctx, cudaEventRecord(e0, st), "event");
                    for (int r = 0; r < 3; ++r) launch();
                    ck(ctx, cudaEventRecord(e1, st), "event");
                    ck(ctx, cudaEventSynchronize(e1), "tuner");
                    ctx->launches += 4;
                    float ms = 0.f;
                    ck(ctx, cudaEventElapsedTime(&ms, e0, e1), "tuner");
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = c;
                    }
                }
                if (digits) ctx->tc_widths[shape_key(sh.M, sh.N, sh.K, sh.nprod, sh.combine) ^ dkey] = best;
                else ctx->gemm_units[shape_key(sh.M, sh.N, sh.K, sh.nprod, sh.combine)] = best;
            }
        } catch (Fail&) {
            ctx->evfree.push_back(e0);
            ctx->evfree.push_back(e1);
            dev_free(ctx, buf);
            throw;
        }
        ctx->evfree.push_back(e0);
        ctx->evfree.push_back(e1);
        dev_free(ctx, buf);
    }

    // ---------------------------------------------------------------- launches
    // Kmax: the largest K of the products (a host-known input or initial-guess rank).
    void gemm(aci::GemmArgs<T>& g, int Mmax, int Nmax, int Kmax, const char* what, int cls) {
        g.chi = chi;
        g.flops = flops_of(cls);
        g.part = gpart;
        g.tile_count = gcount;
        g.target_units = aci::gemm_target_units(ctx->num_sms, units_per_sm(Mmax, Nmax, Kmax, g.nprod, g.combine));
        // On the side stream a pivot search holds up to 16 SMs (its CTAs take nearly the whole
        // register file): a persistent grid over all SMs would leave ~32 of its CTAs waiting for
        // the search to end, each holding a fixed share of the units, so the contraction would
        // take two rounds. Its grid covers only the SMs the search leaves free.
        g.num_sms = (ctx->side && st == ctx->side) ? std::max(1, ctx->num_sms - side_reserve()) : ctx->num_sms;
        cudaEvent_t e = pre(cls);
        if (digits) {
            ck(ctx, aci::launch_gemm_tc<T>(g, Mmax, Nmax, Kmax, digits, tcbuf, tc_bytes, err,
                                           prof ? kflops + 4 + cls : nullptr, st, ctx->pipeline_polls,
                                           tc_width(Mmax, Nmax, Kmax, g.nprod, g.combine)),
               what);
            ctx->launches++;  // digit split + tensor-core contraction
            kcount[cls]++;
        } else {
            aci::launch_gemm<T>(g, Mmax, Nmax, st);
        }
        post(cls, e, what);
    }
    int kmax_of(int s) const {  // largest input rank at bond position s
        int k = 1;
        for (int n = 0; n < N; ++n) k = std::max(k, r[n][s]);
        return k;
    }

    aci::GemmArgs<T> gemm_base() {
        aci::GemmArgs<T> g;
        std::memset(&g, 0, sizeof(g));
        g.op = op;
        return g;
    }

    void prrlu(const T* Min, DimE m, DimE n, int mm, int nn, int out_idx, int b_store, bool with_lu,
               double* eps_out, const unsigned long long* S) {
        aci::PrrluArgs<T> a;
        std::memset(&a, 0, sizeof(a));
        a.Min = Min;
        a.m = m;
        a.n = n;
        a.chi = chi;
        a.chimax = chimax;
        a.out_chi_idx = out_idx;
        a.eps_out = eps_out;
        a.piv_rows = prow[b_store];
        a.piv_cols = pcol[b_store];
        a.D = D[b_store];
        if (with_lu || rook) {  // the rook search keeps its factors: they form its residuals
            a.L = Lm[b_store];
            a.Lld = mcap[b_store];
            a.U = Um[b_store];
            a.Uld = ncap[b_store];
        }
        a.rook = rook;
        a.no_coop = no_coop;
        a.spin_limit = ctx->exchange_polls;
        a.tol = tol;
        a.rel = rel;
        a.smax = S;
        a.W = W;
        a.ll = ll;
        a.tagbase = next_tagbase();
        a.mmax = mm;
        a.nmax = nn;
        a.err = err;
        a.flops = flops_of(ACI_KCLASS_PIVOT);
        const int G = rook ? aci::prrlu_rook_grid(mm, nn, ctx->num_sms) : aci::prrlu_grid(mm, nn, ctx->num_sms);
        cudaEvent_t e = pre(ACI_KCLASS_PIVOT);
        ck(ctx, aci::launch_prrlu<T>(a, G, st), "prrlu launch");
        post(ACI_KCLASS_PIVOT, e, "prrlu");
    }

    // Copy the pivots just stored for bond b (rank chi[kidx]) into history slot `slot` (>= 0), or
    // into the current iteration's half-sweep `half` (slot < 0).
    void hist(int b, int kidx, int slot, int half) {
        if (!hist_on) return;
        aci::HistArgs h;
        h.chi = chi;
        h.kidx = kidx;
        h.prow = prow[b];
        h.pcol = pcol[b];
        h.b = b;
        h.nb = L - 1;
        h.kstride = chimax;
        h.nslots = hist_slots;
        h.slot = slot;
        h.half = half;
        h.iter = hist_iter;
        h.rank = hist_rank;
        h.rows = hist_rows;
        h.cols = hist_cols;
        cudaEvent_t e = pre(ACI_KCLASS_OTHER);
        aci::launch_hist(h, st);
        post(ACI_KCLASS_OTHER, e, "pivot history");
    }

    // Pi[b] = f(LX[.][b] XR[.][b+1]) with the running max |Pi| (Eq. (pifromframes)).
    void pi_block(int b) {
        aci::GemmArgs<T> g = gemm_base();
        g.combine = 1;
        g.nprod = N;
        for (int n = 0; n < N; ++n) {
            g.A[n] = (b == 0) ? Xp(n, 0) : LX[n][b];
            g.B[n] = (b + 1 == L - 1) ? Xp(n, L - 1) : XR[n][b + 1];
            g.K[n] = dimc(r[n][b + 1]);
            g.lda[n] = dimc(r[n][b + 1]);
            g.ldb[n] = dimr(d[b + 1], b + 2);
        }
        g.M[0] = dimr(d[b], b);
        g.N[0] = dimr(d[b + 1], b + 2);
        g.C[0] = Pi[b];
        g.smax = smax;
        gemm(g, mcap[b], ncap[b], kmax_of(b + 1), "pi_block", ACI_KCLASS_PI);
    }

    // Candidate features of bond b (the proposer's inputs), from the operands of its Pi block.
    void features(int b) {
        aci::ProposerArgs<T> a;
        std::memset(&a, 0, sizeof(a));
        for (int n = 0; n < N; ++n) {
            a.A[n] = (b == 0) ? Xp(n, 0) : LX[n][b];
            a.B[n] = (b + 1 == L - 1) ? Xp(n, L - 1) : XR[n][b + 1];
            a.K[n] = dimc(r[n][b + 1]);
            a.lda[n] = dimc(r[n][b + 1]);
            a.ldb[n] = dimr(d[b + 1], b + 2);
        }
        a.M = dimr(d[b], b);
        a.N = dimr(d[b + 1], b + 2);
        a.chi = chi;
        a.nprod = N;
        a.d_row = d[b];
        a.d_col = d[b + 1];
        a.chi_row = dimr(1, b);
        a.chi_col = dimr(1, b + 2);
        a.prev_rows = prow[b];
        a.prev_cols = pcol[b];
        a.kprev = dimr(1, b + 1);
        a.bond_frac = L > 2 ? (float)b / (float)(L - 2) : 0.f;
        a.X = pfeat;
        a.mcap = mcap[b];
        a.ncap = ncap[b];
        cudaEvent_t e = pre(ACI_KCLASS_OTHER);
        a.side_max = pside;
        aci::launch_features<T>(a, st);
        ctx->launches++;  // the norm pass and the finishing pass
        kcount[ACI_KCLASS_OTHER]++;
        post(ACI_KCLASS_OTHER, e, "proposer features");
    }

    // The learned restriction of bond b: scores, kept rows/columns, Pi on them, prrLU, pivots mapped back.
    void proposed_update(int b) {
        features(b);
        cudaEvent_t e = pre(ACI_KCLASS_OTHER);
        aci::launch_mlp_forward(mcap[b] + ncap[b], aci::kPropFeatures, pfeat, ctx->prop_params, 1, pscore, nullptr,
                                nullptr, st);
        aci::TopkArgs t;
        t.z = pscore;
        t.M = dimr(d[b], b);
        t.N = dimr(d[b + 1], b + 2);
        t.kprev = dimr(1, b + 1);
        t.chi = chi;
        t.mcap = mcap[b];
        t.ncap = ncap[b];
        t.keep = ctx->prop_keep;
        t.sel_rows = psel_rows;
        t.sel_cols = psel_cols;
        t.slot_rows = L + 1;
        t.slot_cols = L + 2;
        ck(ctx, aci::launch_topk(t, st), "proposer top-k");
        ctx->launches++;
        kcount[ACI_KCLASS_OTHER]++;
        post(ACI_KCLASS_OTHER, e, "proposer score");
        // Pi on the kept rows and columns (the same contraction, gathered on load)
        aci::GemmArgs<T> g = gemm_base();
        g.combine = 1;
        g.nprod = N;
        for (int n = 0; n < N; ++n) {
            g.A[n] = (b == 0) ? Xp(n, 0) : LX[n][b];
            g.B[n] = (b + 1 == L - 1) ? Xp(n, L - 1) : XR[n][b + 1];
            g.K[n] = dimc(r[n][b + 1]);
            g.lda[n] = dimc(r[n][b + 1]);
            g.ldb[n] = dimr(d[b + 1], b + 2);
        }
        g.arow = psel_rows;
        g.bcol = psel_cols;
        g.M[0] = dimr(1, L + 1);
        g.N[0] = dimr(1, L + 2);
        g.C[0] = Pi[b];
        g.smax = smax;
        gemm(g, mcap[b], ncap[b], kmax_of(b + 1), "pi_block (proposed)", ACI_KCLASS_PI);
        prrlu(Pi[b], dimr(1, L + 1), dimr(1, L + 2), mcap[b], ncap[b], b + 1, b, false, eps_lr + b, smax);
        cudaEvent_t e2 = pre(ACI_KCLASS_OTHER);
        aci::launch_map_pivots(chi, b + 1, prow[b], pcol[b], psel_rows, psel_cols, st);
        post(ACI_KCLASS_OTHER, e2, "proposer map");
        hist(b, b + 1, -1, 0);
    }

    void record(int b) {
        aci::RecordArgs rr;
        rr.X = pfeat;
        rr.M = dimr(d[b], b);
        rr.N = dimr(d[b + 1], b + 2);
        rr.k = dimr(1, b + 1);
        rr.chi = chi;
        rr.mcap = mcap[b];
        rr.prow = prow[b];
        rr.pcol = pcol[b];
        rr.buf = ctx->rec_buf;
        rr.capacity = ctx->rec_cap;
        rr.count = ctx->rec_count;
        cudaEvent_t e = pre(ACI_KCLASS_OTHER);
        aci::launch_record(rr, st);
        post(ACI_KCLASS_OTHER, e, "proposer record");
    }

    // LX[n][b] = rows prow[b-1] of LX[n][b-1], times X^n_b (Leftframe of Algorithm 5).
    void left_half(int b) {
        if (b == 0) return;
        aci::GemmArgs<T> g = gemm_base();
        g.combine = 0;
        g.nprod = N;
        int nmax = 1;
        for (int n = 0; n < N; ++n) {
            g.A[n] = (b - 1 == 0) ? Xp(n, 0) : LX[n][b - 1];
            g.B[n] = Xp(n, b);
            g.C[n] = LX[n][b];
            g.M[n] = dimr(1, b);
            g.N[n] = dimc(d[b] * r[n][b + 1]);
            g.K[n] = dimc(r[n][b]);
            g.lda[n] = dimc(r[n][b]);
            g.ldb[n] = dimc(d[b] * r[n][b + 1]);
            nmax = std::max(nmax, d[b] * r[n][b + 1]);
        }
        g.arow = prow[b - 1];
        gemm(g, cap[b], nmax, kmax_of(b), "left_half", ACI_KCLASS_FRAME);
    }

    // XR[n][s] = X^n_s times columns pcol[s] of XR[n][s+1] (Rightframe of Algorithm 5).
    void right_half(int s) {
        if (s >= L - 1) return;
        aci::GemmArgs<T> g = gemm_base();
        g.combine = 0;
        g.nprod = N;
        int mmax = 1;
        for (int n = 0; n < N; ++n) {
            g.A[n] = Xp(n, s);
            g.B[n] = (s + 1 == L - 1) ? Xp(n, L - 1) : XR[n][s + 1];
            g.C[n] = XR[n][s];
            g.M[n] = dimc(r[n][s] * d[s]);
            g.N[n] = dimr(1, s + 1);
            g.K[n] = dimc(r[n][s + 1]);
            g.lda[n] = dimc(r[n][s + 1]);
            g.ldb[n] = dimr(d[s + 1], s + 2);
            mmax = std::max(mmax, r[n][s] * d[s]);
        }
        g.bcol = pcol[s];
        gemm(g, mmax, cap[s + 1], kmax_of(s + 1), "right_half", ACI_KCLASS_FRAME);
    }

    // ---------------------------------------------------------------- overlapped schedule
    // Left to right, bond b >= 1 needs the rows prow[b-1] of Q^n_b = LX^n_{b-1} X^n_b (every row
    // of Pi[b-1], each a d_b x r_{b+1} block) and the same rows of f(Q_b XR_{b+1}): both are
    // computed on the side stream during the pivot search of bond b-1 and gathered after it.
    // Right to left, bond b needs the columns pcol[b+1] of X_{b+1} XR_{b+2} (every column of
    // Pi[b+1], per sigma_{b+1}) and of f(LX_b X_{b+1} XR_{b+2}), likewise.
    void fork() {  // the side stream waits for the context stream's work so far
        ck(ctx, cudaEventRecord(ctx->ev_fork, st), "fork");
        ck(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0), "fork");
    }
    void join() {  // the context stream waits for the side stream's work so far
        ck(ctx, cudaEventRecord(ctx->ev_join, ctx->side), "join");
        ck(ctx, cudaStreamWaitEvent(st, ctx->ev_join, 0), "join");
    }
    struct OnSide {  // launches (and their timing events) go to the side stream while alive
        Run* r;
        cudaStream_t keep;
        explicit OnSide(Run* rr) : r(rr), keep(rr->st) { r->st = r->ctx->side; }
        ~OnSide() { r->st = keep; }
    };

    // Q^n_{b} over every row of Pi[b-1], then Pfull = f(Q_b XR_{b+1}) (rows: Pi[b-1] rows x d_b).
    void side_lr(int b) {
        OnSide on(this);
        aci::GemmArgs<T> g = gemm_base();
        g.combine = 0;
        g.nprod = N;
        int nmax = 1;
        for (int n = 0; n < N; ++n) {
            g.A[n] = (b - 1 == 0) ? Xp(n, 0) : LX[n][b - 1];
            g.B[n] = Xp(n, b);
            g.C[n] = Qb[n];
            g.M[n] = dimr(d[b - 1], b - 1);
            g.N[n] = dimc(d[b] * r[n][b + 1]);
            g.K[n] = dimc(r[n][b]);
            g.lda[n] = dimc(r[n][b]);
            g.ldb[n] = dimc(d[b] * r[n][b + 1]);
            nmax = std::max(nmax, d[b] * r[n][b + 1]);
        }
        gemm(g, mcap[b - 1], nmax, kmax_of(b), "left_half (all rows)", ACI_KCLASS_FRAME);
        aci::GemmArgs<T> p = gemm_base();
        p.combine = 1;
        p.nprod = N;
        for (int n = 0; n < N; ++n) {
            p.A[n] = Qb[n];
            p.B[n] = (b + 1 == L - 1) ? Xp(n, L - 1) : XR[n][b + 1];
            p.K[n] = dimc(r[n][b + 1]);
            p.lda[n] = dimc(r[n][b + 1]);
            p.ldb[n] = dimr(d[b + 1], b + 2);
        }
        p.M[0] = dimr(d[b - 1] * d[b], b - 1);
        p.N[0] = dimr(d[b + 1], b + 2);
        p.C[0] = Pfull;
        gemm(p, mcap[b - 1] * d[b], ncap[b], kmax_of(b + 1), "pi_block (all rows)", ACI_KCLASS_PI);
    }

    // P^n = X^n_{b+1} XR^n_{b+2} over every column of Pi[b+1], then Pfull = f(LX_b P).
    void side_rl(int b) {
        OnSide on(this);
        aci::GemmArgs<T> g = gemm_base();
        g.combine = 0;
        g.nprod = N;
        int mmax = 1;
        for (int n = 0; n < N; ++n) {
            g.A[n] = Xp(n, b + 1);
            g.B[n] = (b + 2 == L - 1) ? Xp(n, L - 1) : XR[n][b + 2];
            g.C[n] = Qb[n];
            g.M[n] = dimc(r[n][b + 1] * d[b + 1]);
            g.N[n] = dimr(d[b + 2], b + 3);
            g.K[n] = dimc(r[n][b + 2]);
            g.lda[n] = dimc(r[n][b + 2]);
            g.ldb[n] = dimr(d[b + 2], b + 3);
            mmax = std::max(mmax, r[n][b + 1] * d[b + 1]);
        }
        gemm(g, mmax, ncap[b + 1], kmax_of(b + 2), "right_half (all columns)", ACI_KCLASS_FRAME);
        aci::GemmArgs<T> p = gemm_base();
        p.combine = 1;
        p.nprod = N;
        for (int n = 0; n < N; ++n) {
            p.A[n] = (b == 0) ? Xp(n, 0) : LX[n][b];
            p.B[n] = Qb[n];
            p.K[n] = dimc(r[n][b + 1]);
            p.lda[n] = dimc(r[n][b + 1]);
            p.ldb[n] = dimr(d[b + 1] * d[b + 2], b + 3);
        }
        p.M[0] = dimr(d[b], b);
        p.N[0] = dimr(d[b + 1] * d[b + 2], b + 3);
        p.C[0] = Pfull;
        gemm(p, mcap[b], d[b + 1] * ncap[b + 1], kmax_of(b + 1), "pi_block (all columns)", ACI_KCLASS_PI);
    }

    // Pi[b] and LX^n_b: rows prow[b-1] of Pfull and of Q^n_b; max |Pi[b]| into the running max.
    void gather_lr(int b) {
        aci::GatherArgs<T> a;
        std::memset(&a, 0, sizeof(a));
        a.chi = chi;
        a.smax = smax;
        a.smax_job = 0;
        a.njobs = 1 + N;
        aci::GatherJob<T>& pj = a.job[0];
        pj.src = Pfull;
        pj.dst = Pi[b];
        pj.rows = dimr(d[b], b);
        pj.cols = pj.sld = pj.dld = dimr(d[b + 1], b + 2);
        pj.ridx = prow[b - 1];
        pj.rblk = d[b];
        long long mx = (long long)mcap[b] * ncap[b];
        for (int n = 0; n < N; ++n) {
            aci::GatherJob<T>& j = a.job[1 + n];
            j.src = Qb[n];
            j.dst = LX[n][b];
            j.rows = dimr(1, b);
            j.cols = j.sld = j.dld = dimc(d[b] * r[n][b + 1]);
            j.ridx = prow[b - 1];
            mx = std::max(mx, (long long)cap[b] * d[b] * r[n][b + 1]);
        }
        cudaEvent_t e = pre(ACI_KCLASS_OTHER);
        aci::launch_gather<T>(a, mx, ctx->num_sms, st);
        post(ACI_KCLASS_OTHER, e, "gather (left to right)");
    }

    // Pi[b] and XR^n_{b+1}: columns pcol[b+1] (per sigma_{b+1}) of Pfull and of P^n.
    void gather_rl(int b) {
        aci::GatherArgs<T> a;
        std::memset(&a, 0, sizeof(a));
        a.chi = chi;
        a.smax = smax;
        a.smax_job = 0;
        a.njobs = 1 + N;
        auto cols_of = [&](aci::GatherJob<T>& j) {
            j.cols = j.dld = dimr(d[b + 1], b + 2);
            j.sld = dimr(d[b + 1] * d[b + 2], b + 3);
            j.cidx = pcol[b + 1];
            j.cblk = dimr(1, b + 2);
            j.cstride = dimr(d[b + 2], b + 3);
        };
        aci::GatherJob<T>& pj = a.job[0];
        pj.src = Pfull;
        pj.dst = Pi[b];
        pj.rows = dimr(d[b], b);
        cols_of(pj);
        long long mx = (long long)mcap[b] * ncap[b];
        for (int n = 0; n < N; ++n) {
            aci::GatherJob<T>& j = a.job[1 + n];
            j.src = Qb[n];
            j.dst = XR[n][b + 1];
            j.rows = dimc(r[n][b + 1]);
            cols_of(j);
            mx = std::max(mx, (long long)r[n][b + 1] * ncap[b]);
        }
        cudaEvent_t e = pre(ACI_KCLASS_OTHER);
        aci::launch_gather<T>(a, mx, ctx->num_sms, st);
        post(ACI_KCLASS_OTHER, e, "gather (right to left)");
    }

    void ensure_side() {
        if (ctx->side) return;
        ck(ctx, cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking), "side stream");
        ck(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming), "event");
        ck(ctx, cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming), "event");
    }

    // ---------------------------------------------------------------- Algorithm 1
    aci_status run(aci_tt* out, aci_stats* stats, int out_memory) {
        plan_sizes();
        Carver sizer;
        layout(sizer);
        Carver carver;
        carver.base = workspace(ctx, sizer.off);
        layout(carver);
        for (int n = 0; n < N; ++n) {
            Xv[n].assign(L, nullptr);
            for (int s = 0; s < L; ++s) {
                const size_t cnt = (size_t)r[n][s] * d[s] * r[n][s + 1];
                if (host_in) {
                    ck(ctx, cudaMemcpyAsync(Xcopy[n][s], in[n]->core[s], cnt * sizeof(T), cudaMemcpyHostToDevice, st), "copy input");
                    Xv[n][s] = Xcopy[n][s];
                } else {
                    Xv[n][s] = static_cast<const T*>(in[n]->core[s]);
                }
            }
        }
        ck(ctx, cudaEventRecord(ctx->ev0, st), "event");
        const long long launches0 = ctx->launches;
        const int nb = L - 1;

        // constants and per-call state
        std::vector<int> chi_h(L + 3, 0);
        chi_h[0] = 1;
        chi_h[L] = 1;
        ck(ctx, cudaMemcpyAsync(chi, chi_h.data(), sizeof(int) * (L + 3), cudaMemcpyHostToDevice, st), "init chi");
        ck(ctx, cudaMemcpyAsync(dd, d.data(), sizeof(int) * L, cudaMemcpyHostToDevice, st), "init d");
        ck(ctx, cudaMemsetAsync(err, 0, sizeof(int), st), "memset");
        ck(ctx, cudaMemsetAsync(smax, 0, sizeof(unsigned long long), st), "memset");
        ck(ctx, cudaMemsetAsync(kflops, 0, 8 * sizeof(double), st), "memset");
        ck(ctx, cudaMemsetAsync(ll, 0, ll_words * sizeof(unsigned long long), st), "clear exchange");
        prrlu_launches = 0;
        ck(ctx, cudaMemsetAsync(gcount, 0, gcount_n * sizeof(int), st), "clear counters");
        if (autotune) tune_contractions();
        if (hist_on) {  // -1 marks updates that never ran
            ck(ctx, cudaMemsetAsync(hist_rank, 0xFF, sizeof(int) * hist_slots * nb, st), "history");
            ck(ctx, cudaMemsetAsync(hist_rows, 0xFF, sizeof(int) * (size_t)hist_slots * nb * chimax, st), "history");
            ck(ctx, cudaMemsetAsync(hist_cols, 0xFF, sizeof(int) * (size_t)hist_slots * nb * chimax, st), "history");
            ck(ctx, cudaMemsetAsync(hist_iter, 0, sizeof(int), st), "history");
        }
        if (pside) {  // the features' side maxima start empty; every features call leaves them so
            static const int kEmpty[4] = {INT_MIN, INT_MIN, INT_MIN, INT_MIN};
            ck(ctx, cudaMemcpyAsync(pside, kEmpty, sizeof(kEmpty), cudaMemcpyHostToDevice, st), "init side maxima");
        }
        T one_h;
        std::memset(&one_h, 0, sizeof(T));
        *reinterpret_cast<double*>(&one_h) = 1.0;
        ck(ctx, cudaMemcpyAsync(ones, &one_h, sizeof(T), cudaMemcpyHostToDevice, st), "ones");
        if (nb > 0) {
            std::vector<aci::BondBuf<T>> bb(nb);
            std::vector<int*> pc(nb), jp(nb);
            for (int b = 0; b < nb; ++b) {
                bb[b].Pi = Pi[b];
                bb[b].prow = prow[b];
                bb[b].pcol = pcol[b];
                bb[b].D = D[b];
                bb[b].Lm = Lm[b];
                bb[b].Um = Um[b];
                bb[b].Lld = mcap[b];
                bb[b].Uld = ncap[b];
                pc[b] = pcol[b];
                jp[b] = jprev[b];
            }
            ck(ctx, cudaMemcpyAsync(bonds_dev, bb.data(), sizeof(bb[0]) * nb, cudaMemcpyHostToDevice, st), "bonds");
            ck(ctx, cudaMemcpyAsync(pcol_dev, pc.data(), sizeof(int*) * nb, cudaMemcpyHostToDevice, st), "pcol");
            ck(ctx, cudaMemcpyAsync(jprev_dev, jp.data(), sizeof(int*) * nb, cudaMemcpyHostToDevice, st), "jprev");
            ck(ctx, cudaMemcpyAsync(Yptr_dev, Ysc.data(), sizeof(T*) * L, cudaMemcpyHostToDevice, st), "Yptr");
        }

        if (L == 1) {  // no bond: y = f(x) on the single site
            aci::GemmArgs<T> g = gemm_base();
            g.combine = 1;
            g.nprod = N;
            for (int n = 0; n < N; ++n) {
                g.A[n] = Xp(n, 0);
                g.B[n] = ones;
                g.K[n] = dimc(1);
                g.lda[n] = dimc(1);
                g.ldb[n] = dimc(1);
            }
            g.M[0] = dimc(d[0]);
            g.N[0] = dimc(1);
            g.C[0] = Ysc[0];
            g.smax = smax;
            gemm(g, d[0], 1, 1, "single_site", ACI_KCLASS_PI);
            return finish(out, stats, out_memory, 0, 1, 0, launches0);
        }

        // ---- initial guess: counter-based random TT, or the caller's warm start
        if (init) {
            for (int s = 0; s < L; ++s) {
                const size_t cnt = (size_t)ry[s] * d[s] * ry[s + 1];
                const cudaMemcpyKind kind = init->memory == ACI_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
                ck(ctx, cudaMemcpyAsync(Yinit[s], init->core[s], cnt * sizeof(T), kind, st), "copy init");
            }
        } else {
            std::vector<long long> off(L), cnt(L);
            long long o = 0;
            for (int s = 0; s < L; ++s) {
                cnt[s] = (long long)ry[s] * d[s] * ry[s + 1];
                off[s] = o;
                o += cnt[s];
            }
            cudaEvent_t e = pre(ACI_KCLASS_OTHER);
            aci::launch_tt_random<T>(seed, L, off.data(), cnt.data(), Yinit.data(), st);
            ctx->launches += L - 1;
            kcount[ACI_KCLASS_OTHER] += L - 1;
            post(ACI_KCLASS_OTHER, e, "tt_random");
        }

        // ---- CI-canonicalise Y^init right to left; build the right frames (Algorithm 1)
        for (int s = L - 1; s >= 1; --s) {
            T* Ms = Minit[s & 1];
            ck(ctx, cudaMemsetAsync(initmax, 0, sizeof(unsigned long long), st), "memset");
            aci::GemmArgs<T> g = gemm_base();
            g.combine = 0;
            g.nprod = 1;
            g.A[0] = Yinit[s];
            g.C[0] = Ms;
            g.M[0] = dimc(ry[s] * d[s]);
            g.N[0] = dimr(1, s + 1);
            g.K[0] = dimc(ry[s + 1]);
            g.lda[0] = dimc(ry[s + 1]);
            if (s == L - 1) {
                g.B[0] = ones;
                g.ldb[0] = dimc(1);
            } else {
                g.B[0] = Minit[(s + 1) & 1];
                g.ldb[0] = dimr(d[s + 1], s + 2);
                g.bcol = pcol[s];
            }
            g.smax = initmax;
            gemm(g, ry[s] * d[s], cap[s + 1], ry[s + 1], "init_gemm", ACI_KCLASS_OTHER);
            prrlu(Ms, dimc(ry[s]), dimr(d[s], s + 1), ry[s], d[s] * cap[s + 1], s, s - 1, false,
                  eps_junk, initmax);
            hist(s - 1, s, 0, 0);
            right_half(s);
        }
        {
            cudaEvent_t e = pre(ACI_KCLASS_OTHER);
            aci::launch_iter_check(L, chi, chi_prev, pcol_dev, jprev_dev, eps_lr, eps_rl, smax, err, flags, 1, st);
            post(ACI_KCLASS_OTHER, e, "iter_snapshot");
        }

        // ---- sweeps. One iteration (left-to-right and right-to-left sweeps, stop test, flag copy)
        // is enqueued once into a CUDA graph and replayed: every shape is read on the device, so
        // the launches are identical from one iteration to the next. It starts by clearing the
        // pivot-search exchange area, so the tags of its launches are fresh at every replay.
        if (overlap) ensure_side();
        auto enqueue_overlapped = [&]() {
            if (proposed) {
                // the learned restriction keeps the plain left-to-right sweep; its last Pi block
                // is restricted, so the right-to-left sweep starts from the full block
                for (int b = 0; b < nb; ++b) {
                    left_half(b);
                    proposed_update(b);
                }
                pi_block(nb - 1);
                fork();
                side_rl(nb - 2);
            } else {
                // left to right: bond 0 directly, then each bond's Pi gathered from the side stream's work
                pi_block(0);
                fork();
                side_lr(1);
                if (recording) features(0);
                prrlu(Pi[0], dimr(d[0], 0), dimr(d[1], 2), mcap[0], ncap[0], 1, 0, false, eps_lr, smax);
                hist(0, 1, -1, 0);
                if (recording) record(0);
                for (int b = 1; b < nb; ++b) {
                    join();
                    gather_lr(b);
                    fork();
                    if (b + 1 < nb) side_lr(b + 1);
                    else side_rl(nb - 2);  // the first right-to-left work needs no new pivot
                    if (recording) features(b);
                    prrlu(Pi[b], dimr(d[b], b), dimr(d[b + 1], b + 2), mcap[b], ncap[b], b + 1, b, false,
                          eps_lr + b, smax);
                    hist(b, b + 1, -1, 0);
                    if (recording) record(b);
                }
            }
            // right to left: Pi[nb-1] is the full block of the last bond (its frames have not changed)
            prrlu(Pi[nb - 1], dimr(d[nb - 1], nb - 1), dimr(d[nb], nb + 1), mcap[nb - 1], ncap[nb - 1], nb, nb - 1,
                  true, eps_rl + nb - 1, smax);
            hist(nb - 1, nb, -1, 1);
            for (int b = nb - 2; b >= 0; --b) {
                join();
                gather_rl(b);
                if (b > 0) {
                    fork();
                    side_rl(b - 1);
                }
                prrlu(Pi[b], dimr(d[b], b), dimr(d[b + 1], b + 2), mcap[b], ncap[b], b + 1, b, true,
                      eps_rl + b, smax);
                hist(b, b + 1, -1, 1);
            }
        };
        auto enqueue_iteration = [&]() {
            ck(ctx, cudaMemsetAsync(ll, 0, ll_words * sizeof(unsigned long long), st), "clear exchange");
            prrlu_launches = 0;
            if (hist_on) {
                cudaEvent_t e = pre(ACI_KCLASS_OTHER);
                aci::launch_hist_tick(hist_iter, st);
                post(ACI_KCLASS_OTHER, e, "pivot history");
            }
            if (overlap) {
                enqueue_overlapped();
                cudaEvent_t e = pre(ACI_KCLASS_OTHER);
                aci::launch_iter_check(L, chi, chi_prev, pcol_dev, jprev_dev, eps_lr, eps_rl, smax, err, flags, 0, st);
                post(ACI_KCLASS_OTHER, e, "iter_check");
                ck(ctx, cudaMemcpyAsync(ctx->hflags, flags, sizeof(aci::IterFlags), cudaMemcpyDeviceToHost, st), "flags");
                return;
            }
            for (int b = 0; b < nb; ++b) {  // left to right, CI "right"
                left_half(b);
                if (proposed) {  // the learned restriction; the full right-to-left sweep stays the arbiter
                    proposed_update(b);
                    continue;
                }
                if (recording) features(b);
                pi_block(b);
                prrlu(Pi[b], dimr(d[b], b), dimr(d[b + 1], b + 2), mcap[b], ncap[b], b + 1, b, false,
                      eps_lr + b, smax);
                hist(b, b + 1, -1, 0);
                if (recording) record(b);
            }
            for (int b = nb - 1; b >= 0; --b) {  // right to left, CI "left"
                right_half(b + 1);
                pi_block(b);
                prrlu(Pi[b], dimr(d[b], b), dimr(d[b + 1], b + 2), mcap[b], ncap[b], b + 1, b, true,
                      eps_rl + b, smax);
                hist(b, b + 1, -1, 1);
            }
            cudaEvent_t e = pre(ACI_KCLASS_OTHER);
            aci::launch_iter_check(L, chi, chi_prev, pcol_dev, jprev_dev, eps_lr, eps_rl, smax, err, flags, 0, st);
            post(ACI_KCLASS_OTHER, e, "iter_check");
            ck(ctx, cudaMemcpyAsync(ctx->hflags, flags, sizeof(aci::IterFlags), cudaMemcpyDeviceToHost, st), "flags");
        };
        struct GraphGuard {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t e = nullptr;
            ~GraphGuard() {
                if (e) cudaGraphExecDestroy(e);
                if (g) cudaGraphDestroy(g);
            }
        } guard;
        cudaGraph_t& graph = guard.g;
        cudaGraphExec_t& gexec = guard.e;
        long long per_iter_launches = 0;
        long long per_iter_count[4] = {0, 0, 0, 0};
        {
            ck(ctx, cudaStreamSynchronize(st), "before capture");
            harvest();
            const long long l0 = ctx->launches;
            long long c0[4];
            for (int q = 0; q < 4; ++q) c0[q] = kcount[q];
            // relaxed: the first use of a kernel may set its attributes or create events meanwhile
            bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) == cudaSuccess;
            if (ok) {
                try {
                    enqueue_iteration();
                } catch (Fail&) {
                    ok = false;
                }
                cudaError_t e = cudaStreamEndCapture(st, &graph);
                ok = ok && e == cudaSuccess && graph != nullptr;
                if (ok) ok = cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess;
            }
            if (!ok) {  // enqueue directly instead
                cudaGetLastError();
                if (gexec) cudaGraphExecDestroy(gexec);
                if (graph) cudaGraphDestroy(graph);
                gexec = nullptr;
                graph = nullptr;
                for (auto& q : pend) {
                    ctx->evfree.push_back(q.a);
                    ctx->evfree.push_back(q.b);
                }
                pend.clear();
                ctx->err.clear();
            }
            per_iter_launches = ctx->launches - l0;
            for (int q = 0; q < 4; ++q) per_iter_count[q] = kcount[q] - c0[q];
            ctx->launches = l0;
            for (int q = 0; q < 4; ++q) kcount[q] = c0[q];
        }
        int it = 0, converged = 0, fixed = 0;
        aci::IterFlags fl;
        std::memset(&fl, 0, sizeof(fl));
        for (it = 1; it <= maxit; ++it) {
            if (gexec) {
                ck(ctx, cudaGraphLaunch(gexec, st), "graph launch");
                ctx->launches += per_iter_launches;
                for (int q = 0; q < 4; ++q) kcount[q] += per_iter_count[q];
            } else {
                enqueue_iteration();
            }
            ck(ctx, cudaStreamSynchronize(st), "sweep");
            fl = *ctx->hflags;
            harvest(gexec != nullptr);
            if (fl.err & aci::DEVERR_TIMEOUT) fail(ctx, ACI_E_TIMEOUT, "a device-side wait timed out");
            if ((fl.err & aci::DEVERR_NUMERIC) || !(fl.S < INFINITY))
                fail(ctx, ACI_E_NUMERIC, "a non-finite value reached the pivot search");
            const double tau = rel ? tol * fl.S : tol;
            if (!fl.grew && fl.emax <= tau) { converged = 1; break; }
            if (fl.fixed) { fixed = 1; break; }
        }
        if (gexec) {
            for (auto& q : pend) {
                ctx->evfree.push_back(q.a);
                ctx->evfree.push_back(q.b);
            }
            pend.clear();
        }
        if (it > maxit) it = maxit;

        // ---- output: Y_s = T_s P_s^-1 (CI-canonical form)
        aci::AssembleArgs<T> aa;
        aa.L = L;
        aa.chi = chi;
        aa.d = dd;
        aa.bonds = bonds_dev;
        aa.Y = Yptr_dev;
        int Rmax = 1, Kmax = 1;
        for (int s = 0; s < L; ++s) {
            Rmax = std::max(Rmax, cap[s] * d[s]);
            Kmax = std::max(Kmax, cap[s + 1]);
        }
        cudaEvent_t e = pre(ACI_KCLASS_OTHER);
        aci::launch_assemble<T>(aa, Rmax, Kmax, st);
        post(ACI_KCLASS_OTHER, e, "assemble");
        return finish(out, stats, out_memory, it, converged, fixed, launches0, &fl);
    }

    aci_status finish(aci_tt* out, aci_stats* stats, int out_memory, int it, int converged, int fixed,
                      long long launches0, const aci::IterFlags* fl = nullptr) {
        ck(ctx, cudaEventRecord(ctx->ev1, st), "event");
        std::vector<int> chi_h(L + 1, 1);
        if (L > 1) ck(ctx, cudaMemcpyAsync(chi_h.data(), chi, sizeof(int) * (L + 1), cudaMemcpyDeviceToHost, st), "read chi");
        ck(ctx, cudaStreamSynchronize(st), "finish");
        int errflag = 0;
        ck(ctx, cudaMemcpy(&errflag, err, sizeof(int), cudaMemcpyDeviceToHost), "read err");
        if (errflag & aci::DEVERR_TIMEOUT) fail(ctx, ACI_E_TIMEOUT, "a device-side wait timed out");
        if (errflag & aci::DEVERR_NUMERIC) fail(ctx, ACI_E_NUMERIC, "a non-finite value reached the pivot search");
        // allocate and fill the output TT
        int32_t* od = static_cast<int32_t*>(std::malloc(sizeof(int32_t) * L));
        int64_t* orank = static_cast<int64_t*>(std::malloc(sizeof(int64_t) * (L + 1)));
        void** ocore = static_cast<void**>(std::calloc(L, sizeof(void*)));
        if (!od || !orank || !ocore) {
            std::free(od);
            std::free(orank);
            std::free(ocore);
            fail(ctx, ACI_E_ALLOC, "host allocation failed");
        }
        for (int s = 0; s < L; ++s) od[s] = d[s];
        for (int s = 0; s <= L; ++s) orank[s] = chi_h[s];
        try {
            for (int s = 0; s < L; ++s) {
                const size_t cnt = (size_t)orank[s] * d[s] * orank[s + 1];
                if (out_memory == ACI_MEM_HOST) {
                    ocore[s] = std::malloc(std::max<size_t>(cnt * sizeof(T), 1));
                    if (!ocore[s]) fail(ctx, ACI_E_ALLOC, "host allocation failed");
                    ck(ctx, cudaMemcpyAsync(ocore[s], Ysc[s], cnt * sizeof(T), cudaMemcpyDeviceToHost, st), "copy out");
                } else {
                    ocore[s] = dev_alloc(ctx, cnt * sizeof(T));
                    ck(ctx, cudaMemcpyAsync(ocore[s], Ysc[s], cnt * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy out");
                }
            }
            ck(ctx, cudaStreamSynchronize(st), "copy out");
        } catch (Fail&) {
            for (int s = 0; s < L; ++s) {
                if (!ocore[s]) continue;
                if (out_memory == ACI_MEM_HOST) std::free(ocore[s]);
                else dev_free(ctx, ocore[s]);
            }
            std::free(od);
            std::free(orank);
            std::free(ocore);
            throw;
        }
        out->L = L;
        out->dtype = aci::dtype_id<T>::value;
        out->memory = out_memory;
        out->d = od;
        out->rank = orank;
        out->core = ocore;
        if (stats) {
            stats->iterations = it;
            stats->converged = converged;
            stats->fixed_point = fixed;
            stats->L = L;
            stats->scale = fl ? fl->S : 0.0;
            stats->max_eps = fl ? fl->emax : 0.0;
            stats->tau = fl ? (rel ? tol * fl->S : tol) : tol;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            stats->device_ms = ms;
            stats->kernel_launches = ctx->launches - launches0;
            harvest();
            double fl_h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (prof) ck(ctx, cudaMemcpy(fl_h, kflops, sizeof(fl_h), cudaMemcpyDeviceToHost), "flops");
            for (int q = 0; q < 4; ++q) {
                stats->kernel_ms[q] = kms[q];
                stats->kernel_count[q] = kcount[q];
                stats->kernel_flops[q] = fl_h[q];
                stats->tensor_flops[q] = fl_h[4 + q];
            }
            if (stats->ranks)
                for (int s = 0; s <= L; ++s) stats->ranks[s] = chi_h[s];
            if (stats->eps && L > 1) {
                std::vector<double> a(L - 1), b(L - 1);
                ck(ctx, cudaMemcpy(a.data(), eps_lr, sizeof(double) * (L - 1), cudaMemcpyDeviceToHost), "eps");
                ck(ctx, cudaMemcpy(b.data(), eps_rl, sizeof(double) * (L - 1), cudaMemcpyDeviceToHost), "eps");
                for (int q = 0; q < L - 1; ++q) stats->eps[q] = std::max(a[q], b[q]);
            }
            if (hist_on && L > 1) {
                const size_t nr = (size_t)hist_slots * (L - 1);
                ck(ctx, cudaMemcpy(stats->hist_rank, hist_rank, sizeof(int) * nr, cudaMemcpyDeviceToHost), "history");
                ck(ctx, cudaMemcpy(stats->hist_rows, hist_rows, sizeof(int) * nr * chimax, cudaMemcpyDeviceToHost), "history");
                ck(ctx, cudaMemcpy(stats->hist_cols, hist_cols, sizeof(int) * nr * chimax, cudaMemcpyDeviceToHost), "history");
            }
            for (int b = 0; b + 1 < L; ++b) {
                const int k = chi_h[b + 1];
                if (stats->pivot_rows)
                    ck(ctx, cudaMemcpy(stats->pivot_rows + (size_t)b * chimax, prow[b], sizeof(int) * k, cudaMemcpyDeviceToHost), "pivots");
                if (stats->pivot_cols)
                    ck(ctx, cudaMemcpy(stats->pivot_cols + (size_t)b * chimax, pcol[b], sizeof(int) * k, cudaMemcpyDeviceToHost), "pivots");
            }
        }
        return converged || fixed || L == 1 ? ACI_OK : ACI_W_NOT_CONVERGED;
    }
};

void validate_tt(aci_ctx* ctx, const aci_tt* t, const char* name) {
    if (!t->d || !t->rank || !t->core) fail(ctx, ACI_E_ARG, std::string(name) + ": null array");
    if (t->L < 1) fail(ctx, ACI_E_SHAPE, std::string(name) + ": L < 1");
    if (t->L > 4096) fail(ctx, ACI_E_SHAPE, std::string(name) + ": L > 4096");
    if (t->dtype != ACI_R64 && t->dtype != ACI_C128 && t->dtype != ACI_R32 && t->dtype != ACI_C64)
        fail(ctx, ACI_E_DTYPE, std::string(name) + ": unsupported dtype");
    if (t->memory != ACI_MEM_DEVICE && t->memory != ACI_MEM_HOST) fail(ctx, ACI_E_ARG, std::string(name) + ": bad memory kind");
    if (t->rank[0] != 1 || t->rank[t->L] != 1) fail(ctx, ACI_E_SHAPE, std::string(name) + ": rank[0] and rank[L] must be 1");
    for (int s = 0; s < t->L; ++s) {
        if (t->d[s] < 1 || t->d[s] > 4096) fail(ctx, ACI_E_SHAPE, std::string(name) + ": d out of range");
        if (t->rank[s + 1] < 1 || t->rank[s + 1] > (1 << 20)) fail(ctx, ACI_E_SHAPE, std::string(name) + ": rank out of range");
        if (!t->core[s]) fail(ctx, ACI_E_ARG, std::string(name) + ": null core");
    }
}

bool complex_dtype(int dt) { return dt == ACI_C128 || dt == ACI_C64; }

// FP32 / complex64 cores widened to FP64 / complex128 copies in one device buffer (released with
// the object, stream-ordered); FP64 / complex128 TTs pass through untouched.
struct Widened {
    aci_ctx* ctx = nullptr;
    void* buf = nullptr;
    std::vector<void*> core;
    aci_tt tt;
    ~Widened() {
        if (buf) dev_free(ctx, buf);
    }
};

const aci_tt* widen(aci_ctx* ctx, const aci_tt* t, Widened& w) {
    if (!t || (t->dtype != ACI_R32 && t->dtype != ACI_C64)) return t;
    const int L = t->L;
    const size_t per = t->dtype == ACI_C64 ? 2 : 1;  // floats per element
    std::vector<size_t> off(L + 1, 0), cnt(L, 0);
    for (int s = 0; s < L; ++s) {
        cnt[s] = (size_t)t->rank[s] * t->d[s] * t->rank[s + 1] * per;
        off[s + 1] = off[s] + ((cnt[s] + 31) & ~(size_t)31);
    }
    const bool host = t->memory == ACI_MEM_HOST;
    w.ctx = ctx;
    w.buf = dev_alloc(ctx, off[L] * sizeof(double) + (host ? off[L] * sizeof(float) : 0));
    double* dst = static_cast<double*>(w.buf);
    float* stage = host ? reinterpret_cast<float*>(dst + off[L]) : nullptr;
    w.core.assign(L, nullptr);
    for (int s = 0; s < L; ++s) {
        const float* src = static_cast<const float*>(t->core[s]);
        if (host) {
            ck(ctx, cudaMemcpyAsync(stage + off[s], src, cnt[s] * sizeof(float), cudaMemcpyHostToDevice, ctx->stream),
               "copy FP32 input");
            src = stage + off[s];
        }
        aci::launch_promote(src, (long long)cnt[s], dst + off[s], ctx->stream);
        ck(ctx, cudaGetLastError(), "widen FP32 input");
        ctx->launches++;
        w.core[s] = dst + off[s];
    }
    w.tt = *t;
    w.tt.dtype = t->dtype == ACI_C64 ? ACI_C128 : ACI_R64;
    w.tt.memory = ACI_MEM_DEVICE;
    w.tt.core = w.core.data();
    return &w.tt;
}

template <class T>
aci_status run_typed(aci_ctx* ctx, int N, const aci_tt* const* ins, aci_op op, double tol, int32_t max_rank,
                     const aci_opts& o, aci_tt* out, aci_stats* stats) {
    Run<T> R;
    const aci_tt* a = ins[0];
    R.ctx = ctx;
    R.st = ctx->stream;
    R.L = a->L;
    R.N = N;
    for (int n = 0; n < N; ++n) R.in[n] = ins[n];
    R.chimax = max_rank;
    R.tol = tol;
    R.rel = o.tol_kind == ACI_TOL_REL;
    R.maxit = o.max_sweeps;
    R.prof = o.profile ? 1 : 0;
    R.digits = o.precision;
    R.rook = o.pivot_mode == ACI_PIVOT_ROOK ? 1 : 0;
    R.no_coop = ctx->no_coop ? 1 : 0;
    R.proposed = o.pivot_mode == ACI_PIVOT_PROPOSED ? 1 : 0;
    R.overlap_opt = o.sweep_overlap;
    R.recording = ctx->rec_buf != nullptr && !R.proposed && N <= 2;  // the proposer's features take <= 2 inputs
    if (R.proposed && !ctx->prop_params) fail(ctx, ACI_E_ARG, "ACI_PIVOT_PROPOSED needs aci_set_proposer");
    R.seed = o.seed;
    R.hist_on = stats && stats->hist_rank && stats->hist_rows && stats->hist_cols && a->L > 1;
    R.hist_slots = 1 + 2 * o.max_sweeps;
    R.autotune = o.autotune ? 1 : 0;
    R.op = make_op<T>(op);
    R.init = o.init;
    R.host_in = a->memory == ACI_MEM_HOST;
    R.d.assign(a->d, a->d + a->L);
    R.r.assign(R.N, std::vector<int>(a->L + 1));
    for (int n = 0; n < R.N; ++n)
        for (int s = 0; s <= a->L; ++s) R.r[n][s] = (int)R.in[n]->rank[s];
    return R.run(out, stats, o.out_memory);
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

aci_status aci_create(aci_ctx** ctx_out, int device, void* cuda_stream, aci_alloc_fn alloc, aci_free_fn free_fn,
                      void* user) {
    if (!ctx_out) return ACI_E_ARG;
    *ctx_out = nullptr;
    if ((alloc == nullptr) != (free_fn == nullptr)) return ACI_E_ARG;
    aci_ctx* ctx = new (std::nothrow) aci_ctx();
    if (!ctx) return ACI_E_ALLOC;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->user = user;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMallocHost(&ctx->hflags, sizeof(aci::IterFlags)) != cudaSuccess ||
        cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->hflags) cudaFreeHost(ctx->hflags);
        delete ctx;
        return ACI_E_CUDA;
    }
    *ctx_out = ctx;
    return ACI_OK;
}

void aci_destroy(aci_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    for (aci_ctx* w : ctx->workers) aci_destroy(w);
    for (cudaEvent_t e : ctx->worker_ev) cudaEventDestroy(e);
    if (ctx->evb) cudaEventDestroy(ctx->evb);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) dev_free(ctx, ctx->ws);
    if (!ctx->alloc) cudaStreamSynchronize(ctx->stream);
    if (ctx->hflags) cudaFreeHost(ctx->hflags);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (cudaEvent_t e : ctx->evall) cudaEventDestroy(e);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* aci_last_error(const aci_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void aci_opts_default(aci_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol_kind = ACI_TOL_REL;
    o->max_sweeps = 20;
    o->pivot_mode = ACI_PIVOT_FULL;
    o->precision = ACI_PREC_FP64;
    o->seed = 0;
    o->init = nullptr;
    o->out_memory = ACI_MEM_DEVICE;
}

namespace {
// The inputs x^1..x^N of one call (N = 1 for ACI_OP_ABS2_MUL, 2 for the other binary ops, up to
// kMaxInputs for the product of aci_elementwise_n): validation, FP32 widening, dispatch.
aci_status elementwise_inputs(aci_ctx* ctx, int N, const aci_tt* const* ins, aci_op op, double tol, int32_t max_rank,
                              const aci_opts* opts, aci_tt* out, aci_stats* stats) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (!out) fail(ctx, ACI_E_ARG, "out must not be NULL");
        if (N < 1 || N > aci::kMaxInputs) fail(ctx, ACI_E_ARG, "1 to 4 inputs");
        for (int n = 0; n < N; ++n)
            if (!ins[n]) fail(ctx, ACI_E_ARG, n == 0 ? "a must not be NULL" : "b must not be NULL for a binary op");
        if (op.kind < ACI_OP_MUL || op.kind > ACI_OP_AFFINE) fail(ctx, ACI_E_ARG, "unknown op kind");
        if (N > 2 && op.kind != ACI_OP_MUL) fail(ctx, ACI_E_ARG, "more than two inputs: the op must be ACI_OP_MUL");
        if (!(tol >= 0.0) || !(tol < INFINITY)) fail(ctx, ACI_E_ARG, "tol must be finite and >= 0");
        if (max_rank < 1 || max_rank > 8190) fail(ctx, ACI_E_ARG, "max_rank must be in [1, 8190]");
        aci_opts o;
        aci_opts_default(&o);
        if (opts) o = *opts;
        if (o.tol_kind != ACI_TOL_REL && o.tol_kind != ACI_TOL_ABS) fail(ctx, ACI_E_ARG, "bad tol_kind");
        if (o.max_sweeps < 1) fail(ctx, ACI_E_ARG, "max_sweeps must be >= 1");
        if (o.pivot_mode != ACI_PIVOT_FULL && o.pivot_mode != ACI_PIVOT_ROOK && o.pivot_mode != ACI_PIVOT_PROPOSED)
            fail(ctx, ACI_E_ARG, "unsupported pivot mode");
        if (!valid_precision(o.precision)) fail(ctx, ACI_E_ARG, "unsupported precision");
        if (N > 2 && o.precision != ACI_PREC_FP64)
            fail(ctx, ACI_E_ARG, "more than two inputs: the contractions run in FP64 only");
        if (N > 2 && o.pivot_mode == ACI_PIVOT_PROPOSED) fail(ctx, ACI_E_ARG, "the proposer takes at most two inputs");
        if (o.sweep_overlap < ACI_OVERLAP_AUTO || o.sweep_overlap > ACI_OVERLAP_ON)
            fail(ctx, ACI_E_ARG, "unsupported sweep_overlap");
        if (o.out_memory != ACI_MEM_DEVICE && o.out_memory != ACI_MEM_HOST) fail(ctx, ACI_E_ARG, "bad out_memory");
        const aci_tt* a = ins[0];
        validate_tt(ctx, a, "a");
        for (int n = 1; n < N; ++n) {
            const aci_tt* b = ins[n];
            const char* nm = N == 2 ? "b" : "input";
            validate_tt(ctx, b, nm);
            if (b->L != a->L) fail(ctx, ACI_E_SHAPE, N == 2 ? "a and b differ in L" : "the inputs differ in L");
            for (int s = 0; s < a->L; ++s)
                if (a->d[s] != b->d[s]) fail(ctx, ACI_E_SHAPE, N == 2 ? "a and b differ in d" : "the inputs differ in d");
            if (b->dtype != a->dtype) fail(ctx, ACI_E_DTYPE, N == 2 ? "a and b differ in dtype" : "the inputs differ in dtype");
            if (b->memory != a->memory)
                fail(ctx, ACI_E_ARG, N == 2 ? "a and b differ in memory kind" : "the inputs differ in memory kind");
        }
        if (!complex_dtype(a->dtype) && op.kind == ACI_OP_AFFINE)
            for (int i = 0; i < 4; ++i)
                if (op.c[i][1] != 0.0) fail(ctx, ACI_E_DTYPE, "complex coefficients on real inputs");
        if (o.init) {
            validate_tt(ctx, o.init, "init");
            if (o.init->L != a->L || complex_dtype(o.init->dtype) != complex_dtype(a->dtype))
                fail(ctx, ACI_E_SHAPE, "init differs from the inputs");
            for (int s = 0; s < a->L; ++s)
                if (o.init->d[s] != a->d[s]) fail(ctx, ACI_E_SHAPE, "init differs from the inputs in d");
            for (int s = 1; s < a->L; ++s)
                if (o.init->rank[s] > max_rank) fail(ctx, ACI_E_SHAPE, "init ranks exceed max_rank");
        }
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        Widened w[aci::kMaxInputs], wi;
        const aci_tt* X[aci::kMaxInputs] = {};
        for (int n = 0; n < N; ++n) X[n] = widen(ctx, ins[n], w[n]);
        o.init = widen(ctx, o.init, wi);
        if (!complex_dtype(X[0]->dtype)) return run_typed<double>(ctx, N, X, op, tol, max_rank, o, out, stats);
        return run_typed<cplx>(ctx, N, X, op, tol, max_rank, o, out, stats);
    } catch (Fail& f) {
        return f.st;
    } catch (...) {
        ctx->err = "unexpected host exception";
        return ACI_E_ARG;
    }
}
}  // namespace

aci_status aci_elementwise_ex(aci_ctx* ctx, const aci_tt* a, const aci_tt* b, aci_op op, double tol, int32_t max_rank,
                              const aci_opts* opts, aci_tt* out, aci_stats* stats) {
    const aci_tt* ins[2] = {a, b};
    return elementwise_inputs(ctx, op.kind == ACI_OP_ABS2_MUL ? 1 : 2, ins, op, tol, max_rank, opts, out, stats);
}

aci_status aci_elementwise_n(aci_ctx* ctx, int32_t n, const aci_tt* inputs, aci_op op, double tol, int32_t max_rank,
                             const aci_opts* opts, aci_tt* out, aci_stats* stats) {
    if (!ctx) return ACI_E_ARG;
    if (!inputs || n < 1 || n > aci::kMaxInputs) {
        ctx->err = "inputs must hold 1 to 4 TTs";
        return ACI_E_ARG;
    }
    const aci_tt* ins[aci::kMaxInputs] = {};
    for (int i = 0; i < n; ++i) ins[i] = &inputs[i];
    if (n <= 2 && op.kind == ACI_OP_ABS2_MUL && n != 1) {
        ctx->err = "ACI_OP_ABS2_MUL takes one input";
        return ACI_E_ARG;
    }
    if (n == 1 && op.kind != ACI_OP_ABS2_MUL) {
        ctx->err = "one input: the op must be ACI_OP_ABS2_MUL";
        return ACI_E_ARG;
    }
    return elementwise_inputs(ctx, n, ins, op, tol, max_rank, opts, out, stats);
}

aci_status aci_elementwise(aci_ctx* ctx, const aci_tt* a, const aci_tt* b, aci_op op, double tol, int32_t max_rank,
                           aci_tt* out) {
    return aci_elementwise_ex(ctx, a, b, op, tol, max_rank, nullptr, out, nullptr);
}

aci_status aci_elementwise_batch(aci_ctx* ctx, int32_t n, const aci_tt* a, const aci_tt* b, const aci_op* op,
                                 const double* tol, const int32_t* max_rank, const aci_opts* opts, aci_tt* out,
                                 aci_stats* stats, aci_status* status) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (n < 0 || (n > 0 && (!a || !op || !tol || !max_rank || !out))) fail(ctx, ACI_E_ARG, "bad arguments");
        if (n == 0) return ACI_OK;
        aci_opts o;
        aci_opts_default(&o);
        if (opts) o = *opts;
        if (o.init) fail(ctx, ACI_E_ARG, "a batch takes no initial guess");
        if (o.batch_streams < 0) fail(ctx, ACI_E_ARG, "batch_streams must be >= 0");
        if (o.pivot_mode == ACI_PIVOT_ROOK) fail(ctx, ACI_E_ARG, "the rook search is a cooperative grid: not in a batch");
        for (int i = 0; i < n; ++i) std::memset(&out[i], 0, sizeof(aci_tt));
        const int base = std::max(1, ctx->num_sms / 16);  // one pivot-search cluster per product
        aci_ctx::BatchTune* tune = nullptr;
        int W = o.batch_streams;
        if (W == 0) {
            int cls = 0;
            while ((2 << cls) <= n) ++cls;
            tune = &ctx->batch_tune[cls];
            if (tune->cand.empty()) tune->cand = {base, 2 * base, 3 * base};
            W = tune->rate.size() < tune->cand.size() ? tune->cand[tune->rate.size()] : tune->best;
        }
        W = std::min(std::min(W, (int)n), 64);
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        if (!ctx->evb) ck(ctx, cudaEventCreateWithFlags(&ctx->evb, cudaEventDisableTiming), "event");
        while ((int)ctx->workers.size() < W) {
            cudaStream_t sw = nullptr;
            ck(ctx, cudaStreamCreateWithFlags(&sw, cudaStreamNonBlocking), "worker stream");
            aci_ctx* w = nullptr;
            const aci_status cs = aci_create(&w, ctx->device, sw, ctx->alloc, ctx->free_fn, ctx->user);
            if (cs != ACI_OK) {
                cudaStreamDestroy(sw);
                fail(ctx, cs, "worker context creation failed");
            }
            w->own_stream = true;
            w->no_coop = true;
            w->exchange_polls = ctx->exchange_polls;
            w->pipeline_polls = ctx->pipeline_polls;
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                aci_destroy(w);
                fail(ctx, ACI_E_CUDA, "worker event creation failed");
            }
            ctx->workers.push_back(w);
            ctx->worker_ev.push_back(e);
        }
        // the workers start after the context stream's earlier work
        ck(ctx, cudaEventRecord(ctx->evb, ctx->stream), "event");
        for (int w = 0; w < W; ++w) ck(ctx, cudaStreamWaitEvent(ctx->workers[w]->stream, ctx->evb, 0), "stream wait");
        std::atomic<int> next{0};
        std::vector<aci_status> st(n, ACI_OK);
        std::vector<std::string> msg(n);
        auto work = [&](int w) {
            cudaSetDevice(ctx->device);
            aci_ctx* wc = ctx->workers[w];
            for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) {
                st[i] = aci_elementwise_ex(wc, &a[i], b ? &b[i] : nullptr, op[i], tol[i], max_rank[i], &o, &out[i],
                                           stats ? &stats[i] : nullptr);
                if (st[i] < 0) msg[i] = wc->err;
            }
        };
        const auto t0 = std::chrono::steady_clock::now();
        std::vector<std::thread> threads;
        threads.reserve(W);
        for (int w = 1; w < W; ++w) threads.emplace_back(work, w);
        work(0);
        for (auto& t : threads) t.join();
        if (tune && tune->rate.size() < tune->cand.size()) {  // a trial of the autotuner: record its rate
            const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            tune->rate.push_back(n / std::max(sec, 1e-9));
            if (tune->rate.size() == tune->cand.size()) {
                size_t b = 0;
                for (size_t i = 1; i < tune->rate.size(); ++i)
                    if (tune->rate[i] > tune->rate[b]) b = i;
                tune->best = tune->cand[b];
            }
        }
        // the context stream waits for every worker
        for (int w = 0; w < W; ++w) {
            ck(ctx, cudaEventRecord(ctx->worker_ev[w], ctx->workers[w]->stream), "event");
            ck(ctx, cudaStreamWaitEvent(ctx->stream, ctx->worker_ev[w], 0), "stream wait");
        }
        aci_status worst = ACI_OK;
        for (int i = 0; i < n; ++i) {
            if (status) status[i] = st[i];
            if (st[i] < 0 && worst >= 0) {
                worst = st[i];
                ctx->err = "product " + std::to_string(i) + ": " + msg[i];
            } else if (st[i] > 0 && worst == ACI_OK) {
                worst = st[i];
            }
        }
        return worst;
    } catch (Fail& f) {
        return f.st;
    }
}

aci_status aci_tt_release(aci_ctx* ctx, aci_tt* out) {
    if (!ctx || !out) return ACI_E_ARG;
    if (out->core) {
        for (int s = 0; s < out->L; ++s) {
            void* p = const_cast<void*>(out->core[s]);
            if (!p) continue;
            if (out->memory == ACI_MEM_HOST) std::free(p);
            else dev_free(ctx, p);
        }
    }
    std::free(const_cast<void**>(out->core));
    std::free(const_cast<int32_t*>(out->d));
    std::free(const_cast<int64_t*>(out->rank));
    std::memset(out, 0, sizeof(*out));
    return ACI_OK;
}

// ---------------------------------------------------------------- step-level entry points

aci_status aci_k_frame_gemm_prec(aci_ctx* ctx, int32_t dtype, int32_t precision, const void* A, const int32_t* arows,
                                 int32_t M, int32_t K, int32_t lda, const void* B, const int32_t* bcols, int32_t N,
                                 int32_t ldb, void* C) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < K || ldb < 1) fail(ctx, ACI_E_ARG, "bad arguments");
        if (!valid_precision(precision)) fail(ctx, ACI_E_ARG, "unsupported precision");
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        auto go = [&](auto tag) {
            using T = decltype(tag);
            const size_t np = aci::gemm_part_elems(M, N, 1, 0, ctx->num_sms);
            const size_t nc = aci::gemm_tile_counters(M, N, 1);
            aci::TcPlan tp;
            size_t tcb = 0;
            if (precision) {
                tp = aci::tc_plan(precision, sizeof(T) == sizeof(cplx), M, N, K, 1, 0);
                if (!tp.ok) fail(ctx, ACI_E_SHAPE, "contraction too large for the digit-plane precision");
                tcb = aci::tc_scratch_bytes(tp);
            }
            Carver c;
            int *dummy, *cnt, *er;
            T* part;
            unsigned char* tcbuf;
            auto lay = [&](Carver& cv) {
                dummy = cv.take<int>(1);
                er = cv.take<int>(1);
                cnt = cv.take<int>(nc);
                part = cv.take<T>(np);
                tcbuf = cv.take<unsigned char>(tcb);
            };
            lay(c);
            Carver c2;
            c2.base = workspace(ctx, c.off);
            lay(c2);
            ck(ctx, cudaMemsetAsync(cnt, 0, nc * sizeof(int), ctx->stream), "memset");
            ck(ctx, cudaMemsetAsync(er, 0, sizeof(int), ctx->stream), "memset");
            aci::GemmArgs<T> g;
            std::memset(&g, 0, sizeof(g));
            g.part = part;
            g.tile_count = cnt;
            g.target_units = aci::gemm_target_units(ctx->num_sms);
            g.num_sms = ctx->num_sms;
            g.A[0] = static_cast<const T*>(A);
            g.B[0] = static_cast<const T*>(B);
            g.C[0] = static_cast<T*>(C);
            g.M[0] = dimc(M);
            g.N[0] = dimc(N);
            g.K[0] = dimc(K);
            g.lda[0] = dimc(lda);
            g.ldb[0] = dimc(ldb);
            g.arow = arows;
            g.bcol = bcols;
            g.chi = dummy;
            g.nprod = 1;
            if (precision) {
                ck(ctx, aci::launch_gemm_tc<T>(g, M, N, K, precision, tcbuf, tcb, er, nullptr, ctx->stream,
                                               ctx->pipeline_polls),
                   "frame_gemm");
                ctx->launches++;
            } else {
                aci::launch_gemm<T>(g, M, N, ctx->stream);
            }
            note_launch(ctx, "frame_gemm");
            int errflag = 0;
            ck(ctx, cudaMemcpyAsync(&errflag, er, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "err");
            ck(ctx, cudaStreamSynchronize(ctx->stream), "frame_gemm");
            if (errflag & aci::DEVERR_TIMEOUT) fail(ctx, ACI_E_TIMEOUT, "a device-side wait timed out");
        };
        if (dtype == ACI_R64) go(double());
        else if (dtype == ACI_C128) go(cplx());
        else fail(ctx, ACI_E_DTYPE, "unsupported dtype");
        return ACI_OK;
    } catch (Fail& f) {
        return f.st;
    }
}

aci_status aci_k_frame_gemm(aci_ctx* ctx, int32_t dtype, const void* A, const int32_t* arows, int32_t M, int32_t K,
                            int32_t lda, const void* B, const int32_t* bcols, int32_t N, int32_t ldb, void* C) {
    return aci_k_frame_gemm_prec(ctx, dtype, ACI_PREC_FP64, A, arows, M, K, lda, B, bcols, N, ldb, C);
}

aci_status aci_k_pi_block_prec(aci_ctx* ctx, int32_t dtype, int32_t precision, int32_t nprod, const void* const* A,
                               const void* const* B, int32_t M, int32_t N, const int32_t* K, aci_op op, void* Pi,
                               double* maxabs) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (!A || !B || !K || !Pi || M < 1 || N < 1 || nprod < 1 || nprod > 2) fail(ctx, ACI_E_ARG, "bad arguments");
        if (op.kind < ACI_OP_MUL || op.kind > ACI_OP_AFFINE) fail(ctx, ACI_E_ARG, "unknown op kind");
        if (!valid_precision(precision)) fail(ctx, ACI_E_ARG, "unsupported precision");
        int kmax = 1;
        for (int n = 0; n < nprod; ++n) {
            if (K[n] < 1) fail(ctx, ACI_E_ARG, "K must be >= 1");
            kmax = std::max(kmax, (int)K[n]);
        }
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        auto go = [&](auto tag) {
            using T = decltype(tag);
            const size_t np = aci::gemm_part_elems(M, N, nprod, 1, ctx->num_sms);
            const size_t nc = aci::gemm_tile_counters(M, N, nprod);
            aci::TcPlan tp;
            size_t tcb = 0;
            if (precision) {
                tp = aci::tc_plan(precision, sizeof(T) == sizeof(cplx), M, N, kmax, nprod, 1);
                if (!tp.ok) fail(ctx, ACI_E_SHAPE, "contraction too large for the digit-plane precision");
                tcb = aci::tc_scratch_bytes(tp);
            }
            int *dummy, *cnt, *er;
            unsigned long long* smax;
            T* part;
            unsigned char* tcbuf;
            auto lay = [&](Carver& cv) {
                dummy = cv.take<int>(1);
                er = cv.take<int>(1);
                smax = cv.take<unsigned long long>(1);
                cnt = cv.take<int>(nc);
                part = cv.take<T>(np);
                tcbuf = cv.take<unsigned char>(tcb);
            };
            Carver c;
            lay(c);
            Carver c2;
            c2.base = workspace(ctx, c.off);
            lay(c2);
            ck(ctx, cudaMemsetAsync(smax, 0, 8, ctx->stream), "memset");
            ck(ctx, cudaMemsetAsync(er, 0, sizeof(int), ctx->stream), "memset");
            ck(ctx, cudaMemsetAsync(cnt, 0, nc * sizeof(int), ctx->stream), "memset");
            aci::GemmArgs<T> g;
            std::memset(&g, 0, sizeof(g));
            g.part = part;
            g.tile_count = cnt;
            g.target_units = aci::gemm_target_units(ctx->num_sms);
            g.num_sms = ctx->num_sms;
            for (int n = 0; n < nprod; ++n) {
                g.A[n] = static_cast<const T*>(A[n]);
                g.B[n] = static_cast<const T*>(B[n]);
                g.K[n] = dimc(K[n]);
                g.lda[n] = dimc(K[n]);
                g.ldb[n] = dimc(N);
            }
            g.M[0] = dimc(M);
            g.N[0] = dimc(N);
            g.C[0] = static_cast<T*>(Pi);
            g.chi = dummy;
            g.nprod = nprod;
            g.combine = 1;
            g.op = make_op<T>(op);
            g.smax = smax;
            if (precision) {
                ck(ctx, aci::launch_gemm_tc<T>(g, M, N, kmax, precision, tcbuf, tcb, er, nullptr, ctx->stream,
                                               ctx->pipeline_polls),
                   "pi_block");
                ctx->launches++;
            } else {
                aci::launch_gemm<T>(g, M, N, ctx->stream);
            }
            note_launch(ctx, "pi_block");
            unsigned long long bits = 0;
            int errflag = 0;
            ck(ctx, cudaMemcpyAsync(&bits, smax, 8, cudaMemcpyDeviceToHost, ctx->stream), "maxabs");
            ck(ctx, cudaMemcpyAsync(&errflag, er, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "err");
            ck(ctx, cudaStreamSynchronize(ctx->stream), "pi_block");
            if (errflag & aci::DEVERR_TIMEOUT) fail(ctx, ACI_E_TIMEOUT, "a device-side wait timed out");
            if (maxabs) std::memcpy(maxabs, &bits, 8);
        };
        if (dtype == ACI_R64) go(double());
        else if (dtype == ACI_C128) go(cplx());
        else fail(ctx, ACI_E_DTYPE, "unsupported dtype");
        return ACI_OK;
    } catch (Fail& f) {
        return f.st;
    }
}

aci_status aci_k_pi_block(aci_ctx* ctx, int32_t dtype, int32_t nprod, const void* const* A, const void* const* B,
                          int32_t M, int32_t N, const int32_t* K, aci_op op, void* Pi, double* maxabs) {
    return aci_k_pi_block_prec(ctx, dtype, ACI_PREC_FP64, nprod, A, B, M, N, K, op, Pi, maxabs);
}

namespace {
aci_status k_prrlu(aci_ctx* ctx, int rook, int32_t dtype, const void* Min, int32_t m, int32_t n, double tau,
                   int32_t chimax, int32_t* piv_rows, int32_t* piv_cols, void* D, void* L, void* U, int32_t* k_out,
                   double* eps_out) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (!Min || !piv_rows || !piv_cols || !D || !k_out || !eps_out || m < 1 || n < 1 || chimax < 1 ||
            !(tau >= 0.0))
            fail(ctx, ACI_E_ARG, "bad arguments");
        if ((long long)m * n >= (1LL << 31)) fail(ctx, ACI_E_SHAPE, "matrix too large");
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        const int kcap = std::min(std::min(m, n), chimax);
        if (kcap > 8190) fail(ctx, ACI_E_SHAPE, "more than 8190 pivots requested");
        if (rook && kcap > (dtype == ACI_C128 ? 2048 : 4096)) fail(ctx, ACI_E_SHAPE, "too many pivots for the rook search");
        const int G = rook ? aci::prrlu_rook_grid(m, n, ctx->num_sms) : aci::prrlu_grid(m, n, ctx->num_sms);
        auto go = [&](auto tag) {
            using T = decltype(tag);
            const bool cv = sizeof(T) == sizeof(cplx);
            const size_t nll = rook ? aci::prrlu_rook_ll_words(G) : aci::prrlu_ll_words(m, G, cv);
            const size_t nw = rook ? aci::prrlu_rook_scratch_elems(m, n, cv) : (size_t)m * n;
            const bool own_lu = rook && (!L || !U);  // the rook search needs its factors
            Carver c;
            T *Ls = nullptr, *Us = nullptr;
            auto lay = [&](Carver& cv, int** kk, double** ee, int** er, int** chi_d, T** W, unsigned long long** ll) {
                *kk = cv.take<int>(1);
                *ee = cv.take<double>(1);
                *er = cv.take<int>(1);
                *chi_d = cv.take<int>(1);
                *W = cv.take<T>(nw);
                *ll = cv.take<unsigned long long>(nll);
                if (own_lu) {
                    Ls = cv.take<T>((size_t)m * kcap);
                    Us = cv.take<T>((size_t)kcap * n);
                }
            };
            int *kk, *er, *chi_d;
            double* ee;
            T* W;
            unsigned long long* ll;
            lay(c, &kk, &ee, &er, &chi_d, &W, &ll);
            Carver c2;
            c2.base = workspace(ctx, c.off);
            lay(c2, &kk, &ee, &er, &chi_d, &W, &ll);
            ck(ctx, cudaMemsetAsync(er, 0, sizeof(int), ctx->stream), "memset");
            ck(ctx, cudaMemsetAsync(ll, 0, nll * sizeof(unsigned long long), ctx->stream), "clear exchange");
            aci::PrrluArgs<T> a;
            std::memset(&a, 0, sizeof(a));
            a.Min = static_cast<const T*>(Min);
            a.m = dimc(m);
            a.n = dimc(n);
            a.chi = chi_d;
            a.chimax = chimax;
            a.out_chi_idx = -1;
            a.k_out = kk;
            a.eps_out = ee;
            a.piv_rows = piv_rows;
            a.piv_cols = piv_cols;
            a.D = static_cast<T*>(D);
            a.L = own_lu ? Ls : static_cast<T*>(L);
            a.Lld = m;
            a.U = own_lu ? Us : static_cast<T*>(U);
            a.Uld = n;
            a.rook = rook;
            a.spin_limit = ctx->exchange_polls;
            a.tol = tau;
            a.rel = 0;
            a.W = W;
            a.ll = ll;
            a.tagbase = 1u << aci::kPrrluStepBits;
            a.mmax = m;
            a.nmax = n;
            a.err = er;
            ck(ctx, aci::launch_prrlu<T>(a, G, ctx->stream), "prrlu launch");
            note_launch(ctx, "prrlu");
            int errflag = 0;
            ck(ctx, cudaMemcpyAsync(k_out, kk, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "k");
            ck(ctx, cudaMemcpyAsync(eps_out, ee, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "eps");
            ck(ctx, cudaMemcpyAsync(&errflag, er, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "err");
            ck(ctx, cudaStreamSynchronize(ctx->stream), "prrlu");
            if (errflag & aci::DEVERR_TIMEOUT) fail(ctx, ACI_E_TIMEOUT, "pivot search wait timed out");
            if (errflag & aci::DEVERR_NUMERIC) fail(ctx, ACI_E_NUMERIC, "non-finite pivot");
            (void)kcap;
        };
        if (dtype == ACI_R64) go(double());
        else if (dtype == ACI_C128) go(cplx());
        else fail(ctx, ACI_E_DTYPE, "unsupported dtype");
        return ACI_OK;
    } catch (Fail& f) {
        return f.st;
    }
}
}  // namespace

aci_status aci_k_prrlu(aci_ctx* ctx, int32_t dtype, const void* Min, int32_t m, int32_t n, double tau, int32_t chimax,
                       int32_t* piv_rows, int32_t* piv_cols, void* D, void* L, void* U, int32_t* k_out,
                       double* eps_out) {
    return k_prrlu(ctx, 0, dtype, Min, m, n, tau, chimax, piv_rows, piv_cols, D, L, U, k_out, eps_out);
}

aci_status aci_k_prrlu_rook(aci_ctx* ctx, int32_t dtype, const void* Min, int32_t m, int32_t n, double tau,
                            int32_t chimax, int32_t* piv_rows, int32_t* piv_cols, void* D, void* L, void* U,
                            int32_t* k_out, double* eps_out) {
    return k_prrlu(ctx, 1, dtype, Min, m, n, tau, chimax, piv_rows, piv_cols, D, L, U, k_out, eps_out);
}

aci_status aci_set_proposer(aci_ctx* ctx, const float* params, int32_t nfeatures, float keep) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    if (params && nfeatures != aci::kPropFeatures) {
        ctx->err = "the proposer takes " + std::to_string(aci::kPropFeatures) + " features";
        return ACI_E_ARG;
    }
    if (params && !(keep >= 1.0f)) {
        ctx->err = "keep must be >= 1";
        return ACI_E_ARG;
    }
    ctx->prop_params = params;
    ctx->prop_keep = keep;
    return ACI_OK;
}

aci_status aci_set_proposer_record(aci_ctx* ctx, float* buf, int64_t capacity, uint64_t* count) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    if (buf && (capacity < 1 || !count)) {
        ctx->err = "bad arguments";
        return ACI_E_ARG;
    }
    ctx->rec_buf = buf;
    ctx->rec_cap = buf ? capacity : 0;
    ctx->rec_count = buf ? reinterpret_cast<unsigned long long*>(count) : nullptr;
    return ACI_OK;
}

int64_t aci_k_mlp_param_count(int32_t F) {
    return (F >= 1 && F <= aci::kMlpMaxInputs) ? (int64_t)aci::mlp_param_count(F) : -1;
}

aci_status aci_k_mlp_forward(aci_ctx* ctx, int32_t n, int32_t F, const float* X, const float* params,
                             int32_t fp16_weights, float* z) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (n < 0 || F < 1 || F > aci::kMlpMaxInputs || (n > 0 && (!X || !params || !z)))
            fail(ctx, ACI_E_ARG, "bad arguments");
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        aci::launch_mlp_forward(n, F, X, params, fp16_weights ? 1 : 0, z, nullptr, nullptr, ctx->stream);
        note_launch(ctx, "mlp_forward");
        ck(ctx, cudaStreamSynchronize(ctx->stream), "mlp_forward");
        return ACI_OK;
    } catch (Fail& f) {
        return f.st;
    }
}

aci_status aci_k_mlp_grad(aci_ctx* ctx, int32_t n, int32_t F, const float* X, const float* y, float pos_weight,
                          const float* params, float* grad, double* loss) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (n < 1 || F < 1 || F > aci::kMlpMaxInputs || !X || !y || !params || !grad || !loss || !(pos_weight > 0))
            fail(ctx, ACI_E_ARG, "bad arguments");
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        char* ws = workspace(ctx, 256 + sizeof(float) * aci::mlp_train_scratch(n));
        double* dloss = reinterpret_cast<double*>(ws);
        float* scratch = reinterpret_cast<float*>(ws + 256);
        aci::launch_mlp_grad(n, F, X, y, pos_weight, params, grad, dloss, scratch, ctx->stream);
        note_launch(ctx, "mlp_grad");
        ck(ctx, cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "loss");
        ck(ctx, cudaStreamSynchronize(ctx->stream), "mlp_grad");
        return ACI_OK;
    } catch (Fail& f) {
        return f.st;
    }
}

aci_status aci_k_mlp_adam(aci_ctx* ctx, int32_t count, float* params, const float* grad, float* m, float* v,
                          int32_t t, float lr, float beta1, float beta2, float eps) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (count < 0 || t < 1 || (count > 0 && (!params || !grad || !m || !v))) fail(ctx, ACI_E_ARG, "bad arguments");
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        aci::launch_mlp_adam(count, params, grad, m, v, t, lr, beta1, beta2, eps, ctx->stream);
        note_launch(ctx, "mlp_adam");
        ck(ctx, cudaStreamSynchronize(ctx->stream), "mlp_adam");
        return ACI_OK;
    } catch (Fail& f) {
        return f.st;
    }
}

aci_status aci_k_tt_random(aci_ctx* ctx, int32_t dtype, uint64_t seed, int32_t L, const int32_t* d,
                           const int64_t* rank, void* const* cores) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (!d || !rank || !cores || L < 1) fail(ctx, ACI_E_ARG, "bad arguments");
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        std::vector<long long> off(L), cnt(L);
        long long o = 0;
        for (int s = 0; s < L; ++s) {
            cnt[s] = rank[s] * d[s] * rank[s + 1];
            off[s] = o;
            o += cnt[s];
        }
        if (dtype == ACI_R64)
            aci::launch_tt_random<double>(seed, L, off.data(), cnt.data(), reinterpret_cast<double* const*>(cores), ctx->stream);
        else if (dtype == ACI_C128)
            aci::launch_tt_random<cplx>(seed, L, off.data(), cnt.data(), reinterpret_cast<cplx* const*>(cores), ctx->stream);
        else fail(ctx, ACI_E_DTYPE, "unsupported dtype");
        note_launch(ctx, "tt_random");
        ck(ctx, cudaStreamSynchronize(ctx->stream), "tt_random");
        return ACI_OK;
    } catch (Fail& f) {
        return f.st;
    }
}

aci_status aci_k_reciprocal(aci_ctx* ctx, const double* x, int32_t n, double* y) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (!x || !y || n < 1) fail(ctx, ACI_E_ARG, "bad arguments");
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        aci::launch_recip(x, n, y, ctx->stream);
        note_launch(ctx, "reciprocal");
        ck(ctx, cudaStreamSynchronize(ctx->stream), "reciprocal");
        return ACI_OK;
    } catch (Fail& f) {
        return f.st;
    }
}

aci_status aci_set_wait_limits(aci_ctx* ctx, int64_t exchange_polls, int64_t pipeline_polls) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    if (exchange_polls < 0 || pipeline_polls < 0) {
        ctx->err = "wait limits must be >= 0";
        return ACI_E_ARG;
    }
    ctx->exchange_polls = exchange_polls;
    ctx->pipeline_polls = pipeline_polls;
    for (aci_ctx* w : ctx->workers) {
        w->exchange_polls = exchange_polls;
        w->pipeline_polls = pipeline_polls;
    }
    return ACI_OK;
}

aci_status aci_k_fp64_peak(aci_ctx* ctx, int32_t blocks, int32_t iters, double* tflops) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    double* dev = nullptr;
    try {
        if (!tflops || blocks < 1 || blocks > 65535 || iters < 1 || iters > (1 << 24))
            fail(ctx, ACI_E_ARG, "bad arguments");
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        dev = static_cast<double*>(dev_alloc(ctx, sizeof(double) * (2 + (size_t)blocks)));
        const double seed[2] = {1e-3, 0.999999};
        ck(ctx, cudaMemcpyAsync(dev, seed, sizeof(seed), cudaMemcpyHostToDevice, ctx->stream), "probe seed");
        aci::launch_fp64_probe(dev, blocks, iters, dev + 2, ctx->stream);  // warm-up
        note_launch(ctx, "fp64 probe");
        ck(ctx, cudaEventRecord(ctx->ev0, ctx->stream), "event");
        aci::launch_fp64_probe(dev, blocks, iters, dev + 2, ctx->stream);
        note_launch(ctx, "fp64 probe");
        ck(ctx, cudaEventRecord(ctx->ev1, ctx->stream), "event");
        ck(ctx, cudaStreamSynchronize(ctx->stream), "fp64 probe");
        float ms = 0.f;
        ck(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1), "event time");
        *tflops = aci::fp64_probe_flops(blocks, iters) / (ms * 1e-3) / 1e12;
        dev_free(ctx, dev);
        return ACI_OK;
    } catch (Fail& f) {
        if (dev) dev_free(ctx, dev);
        return f.st;
    }
}

aci_status aci_k_apply_pinv(aci_ctx* ctx, int32_t dtype, const void* Tm, int32_t R, int32_t k, const void* LI,
                            const void* D, const void* UJ, void* Y) {
    if (!ctx) return ACI_E_ARG;
    ctx->err.clear();
    try {
        if (!Tm || !LI || !D || !UJ || !Y || R < 1 || k < 1) fail(ctx, ACI_E_ARG, "bad arguments");
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        if (dtype == ACI_R64)
            aci::launch_apply_pinv<double>(static_cast<const double*>(Tm), R, k, static_cast<const double*>(LI),
                                           static_cast<const double*>(D), static_cast<const double*>(UJ),
                                           static_cast<double*>(Y), ctx->stream);
        else if (dtype == ACI_C128)
            aci::launch_apply_pinv<cplx>(static_cast<const cplx*>(Tm), R, k, static_cast<const cplx*>(LI),
                                         static_cast<const cplx*>(D), static_cast<const cplx*>(UJ),
                                         static_cast<cplx*>(Y), ctx->stream);
        else fail(ctx, ACI_E_DTYPE, "unsupported dtype");
        note_launch(ctx, "apply_pinv");
        ck(ctx, cudaStreamSynchronize(ctx->stream), "apply_pinv");
        return ACI_OK;
    } catch (Fail& f) {
        return f.st;
    }
}

}  // extern "C"
