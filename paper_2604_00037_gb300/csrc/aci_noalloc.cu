// Pivot search (rank-revealing LU) for callers that cannot allocate device memory.
//
// Some callers of this library may not allocate: code embedded in a host application that owns
// every byte of device memory and forbids libraries from calling cudaMalloc behind its back,
// code with a fixed, pre-planned memory budget, and code paths where a device allocation is not
// acceptable because it can block on the device or take allocator locks. For them,
// aci_k_prrlu_static runs the same pivot-search kernel as aci_k_prrlu, with its scratch (the
// working copy of the matrix, the per-step records and candidate columns, and a few scalars)
// carved from one file-scope device array instead of the context workspace. The caller passes
// the input and output buffers; the call allocates nothing.
//
// Limits and sharing:
//  * The array is kStaticBytes (8 MiB). Every GPU that loads the library holds it until the
//    process exits. Inputs must satisfy m <= 4096, n <= 4096 and m * n <= 262144; larger
//    shapes are rejected with ACI_E_SHAPE before anything runs. Every shape within these limits
//    runs: the working copy of the matrix takes at most 4 MiB (m n entries of 8 or 16 bytes), and
//    when the block is large enough for the cooperative grid variant (more than 2^18 FP64
//    multiply-adds per step: m n > 2^18 real, > 2^16 complex), its grid is capped so that the
//    exchange words (2 G (8 + m w) words of 8 bytes, w = 2 real / 4 complex) fit in the rest.
//    Such a call may therefore run on fewer CTAs than aci_k_prrlu would (same results, as the
//    pivots and factors do not depend on the grid size).
//  * Every call on a device uses the same array and leaves its contents behind; each call first
//    zeroes what must start at zero (the error flag and the words the CTAs exchange at every
//    pivot step), so stale contents are never read. Calls that overlap on the GPU (two streams,
//    or two host threads at once) race on the array: serialise them.
//  * The first call on each device, with that device current, looks up the array's device
//    address (cudaGetSymbolAddress) and caches it. Make that first call before any stream
//    capture.
#include <cstring>
#include <mutex>

#include "../../include/aci_kernels.h"
#include "aci_internal.h"

namespace {

constexpr size_t kStaticBytes = size_t(8) << 20;
constexpr int kMaxDim = 4096;
constexpr long long kMaxElems = 1LL << 18;
constexpr int kMaxDevices = 64;
// FP64 multiply-adds per pivot step above which the pivot search takes the cooperative grid
// variant (the single-cluster variants use no exchange words); the same bound as launch_prrlu's.
constexpr long long kGridWork = 1LL << 18;

// The scratch. In host code this name is only a host-side stand-in for the symbol: the device
// address comes from cudaGetSymbolAddress in static_scratch() below.
__device__ __align__(256) unsigned char g_prrlu_scratch[kStaticBytes];

struct StaticDevice {
    bool ready = false;
    unsigned char* base = nullptr;
    int num_sms = 0;
};

std::mutex g_static_mu;
StaticDevice g_static_dev[kMaxDevices];

// Once per device (with that device current): resolve and cache the array's device address.
aci_status static_scratch(int dev, unsigned char** base, int* num_sms) {
    if (dev < 0 || dev >= kMaxDevices) return ACI_E_ARG;
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticDevice& s = g_static_dev[dev];
    if (!s.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_prrlu_scratch) != cudaSuccess) {
            cudaGetLastError();
            return ACI_E_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return ACI_E_CUDA;
        }
        s.base = static_cast<unsigned char*>(p);
        s.num_sms = sms;
        s.ready = true;
    }
    *base = s.base;
    *num_sms = s.num_sms;
    return ACI_OK;
}

struct Bump {
    unsigned char* base;
    size_t off = 0;
    template <class U> U* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        U* p = reinterpret_cast<U*>(base + off);
        off += count * sizeof(U);
        return p;
    }
};

template <class T>
aci_status run_static(cudaStream_t st, const void* Min, int m, int n, double tau, int chimax, int32_t* piv_rows,
                      int32_t* piv_cols, void* D, void* L, void* U, int32_t* k_out, double* eps_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return ACI_E_CUDA;
    }
    unsigned char* base = nullptr;
    int sms = 0;
    aci_status s = static_scratch(dev, &base, &sms);
    if (s != ACI_OK) return s;
    const bool cp = sizeof(T) == sizeof(aci::cplx);
    Bump b{base};
    int* k_dev = b.take<int>(1);
    double* eps_dev = b.take<double>(1);
    int* err_dev = b.take<int>(1);
    int* chi_dev = b.take<int>(1);
    T* W = b.take<T>(size_t(m) * n);
    // The exchange words are used by the cooperative grid variant only (blocks of more than
    // kGridWork multiply-adds per step); its grid is capped to what the rest of the array holds.
    int G = 1;
    size_t nll = 0;
    unsigned long long* ll = nullptr;
    if ((long long)m * n * (cp ? 4 : 1) > kGridWork) {
        G = aci::prrlu_grid(m, n, sms);
        const size_t room = kStaticBytes - ((b.off + 255) & ~size_t(255));
        while (G > 1 && aci::prrlu_ll_words(m, G, cp) * sizeof(unsigned long long) > room) --G;
        nll = aci::prrlu_ll_words(m, G, cp);
        ll = b.take<unsigned long long>(nll);
    }
    if (b.off > kStaticBytes) return ACI_E_SHAPE;  // a shape outside the documented limits

    // zero what must start at zero: the error flag and the pivot-search exchange words
    if (cudaMemsetAsync(err_dev, 0, sizeof(int), st) != cudaSuccess ||
        (nll && cudaMemsetAsync(ll, 0, nll * sizeof(unsigned long long), st) != cudaSuccess)) {
        cudaGetLastError();
        return ACI_E_CUDA;
    }
    aci::PrrluArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.Min = static_cast<const T*>(Min);
    a.m = aci::dimc(m);
    a.n = aci::dimc(n);
    a.chi = chi_dev;
    a.chimax = chimax;
    a.out_chi_idx = -1;
    a.k_out = k_dev;
    a.eps_out = eps_dev;
    a.piv_rows = piv_rows;
    a.piv_cols = piv_cols;
    a.D = static_cast<T*>(D);
    a.L = static_cast<T*>(L);
    a.Lld = m;
    a.U = static_cast<T*>(U);
    a.Uld = n;
    a.tol = tau;
    a.rel = 0;
    a.W = W;
    a.ll = ll;
    a.tagbase = 1u << aci::kPrrluStepBits;
    a.mmax = m;
    a.nmax = n;
    a.err = err_dev;
    if (aci::launch_prrlu<T>(a, G, st) != cudaSuccess) {
        cudaGetLastError();
        return ACI_E_CUDA;
    }
    int err = 0;
    if (cudaMemcpyAsync(k_out, k_dev, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(eps_out, eps_dev, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&err, err_dev, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return ACI_E_CUDA;
    }
    if (err & aci::DEVERR_TIMEOUT) return ACI_E_TIMEOUT;
    if (err & aci::DEVERR_NUMERIC) return ACI_E_NUMERIC;
    return ACI_OK;
}

}  // namespace

extern "C" aci_status aci_k_prrlu_static(void* cuda_stream, int32_t dtype, const void* Min, int32_t m, int32_t n,
                                         double tau, int32_t chimax, int32_t* piv_rows, int32_t* piv_cols, void* D,
                                         void* L, void* U, int32_t* k_out, double* eps_out) {
    if (!Min || !piv_rows || !piv_cols || !D || !k_out || !eps_out || m < 1 || n < 1 || chimax < 1 || !(tau >= 0.0))
        return ACI_E_ARG;
    if (m > kMaxDim || n > kMaxDim || (long long)m * n > kMaxElems) return ACI_E_SHAPE;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (dtype == ACI_R64)
        return run_static<double>(st, Min, m, n, tau, chimax, piv_rows, piv_cols, D, L, U, k_out, eps_out);
    if (dtype == ACI_C128)
        return run_static<aci::cplx>(st, Min, m, n, tau, chimax, piv_rows, piv_cols, D, L, U, k_out, eps_out);
    return ACI_E_DTYPE;
}
