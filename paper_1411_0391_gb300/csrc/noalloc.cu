// Allocation-free variant of the truncated SVD (tn_truncated_svd_noalloc).
//
// Some callers cannot allocate device memory at the point where they need the
// projector SVD: a process whose device memory is entirely reserved by another
// allocator (a framework's caching pool), code where the implicit device-wide
// synchronisation of cudaMalloc/cudaFree is not acceptable, or a plugin that is
// not allowed to own device allocations and has no context workspace to lend.
// This entry point takes only the caller's input and output buffers; its
// scratch is the file-scope device array below, of a fixed, modest size
// (TN_NOALLOC_SCRATCH_DOUBLES doubles, 8 MiB), which every GPU that loads the
// library holds until the process exits.
//
// It runs the same implementation as tn_truncated_svd (one-sided Jacobi for
// m <= 112, subspace iteration with Rayleigh-Ritz otherwise) on a view of the
// static array instead of a context workspace.
#include <algorithm>
#include <cmath>
#include "common.cuh"
#include "kernels.cuh"
#include "smallla.cuh"

#define TN_NOALLOC_SCRATCH_DOUBLES (1 << 20)

// Shared by every call on a device; nothing in it is assumed to start at zero
// (each call writes every scratch entry before reading it).
static __device__ __align__(256) double g_noalloc_scratch[TN_NOALLOC_SCRATCH_DOUBLES];

namespace tn {

namespace {

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the symbol is only a stand-in; kernels need the address returned by
// cudaGetSymbolAddress with the device current.  The per-device slots are
// atomics (two host threads may make their first call on one device at the
// same time; both store the same address).  Devices with an index beyond the
// table look the address up on every call.  The cache is not reset-safe: after
// cudaDeviceReset on a device its slot holds the address of the old context.
constexpr int MAX_DEVICES = 64;
std::atomic<double*> g_scratch_addr[MAX_DEVICES];

int scratch_address(double** out)
{
    int dev = 0;
    TN_CUDA(cudaGetDevice(&dev));
    const bool cached = dev >= 0 && dev < MAX_DEVICES;
    double* p = cached ? g_scratch_addr[dev].load(std::memory_order_acquire) : nullptr;
    if (!p) {
        void* a = nullptr;
        TN_CUDA(cudaGetSymbolAddress(&a, g_noalloc_scratch));
        p = static_cast<double*>(a);
        if (cached) g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return TN_OK;
}

// Doubles of scratch the call (m, k) needs: the carving of truncated_svd
// (panels, Ritz blocks, the kk x kk blocks B, Ub, Vb) plus the largest
// temporary inside an iteration (the six kk x kk blocks of the refined Ritz
// SVD; the orthonormalisations take two).  Split-K partial sums are optional:
// when they do not fit, the products run without splitting.
size_t need(int m, int k)
{
    auto al = [](size_t n) { return tn_align256(n * sizeof(double)) / sizeof(double); };
    if (m <= SMALL_MAX) return al((size_t)m * m) * 2 + al(m);
    const int kk = tsvd_columns(m, k);
    return 4 * al((size_t)m * kk) + 2 * al((size_t)m * k) + 9 * al((size_t)kk * kk) + 2 * al(kk);
}

}  // namespace

}  // namespace tn

using namespace tn;

extern "C" int tn_truncated_svd_noalloc(const double* dM, int m, int k, double* dU, double* dS, double* dV,
                                        const double* warm, void* stream)
{
    if (!dM || !dU || !dS || !dV || m < 1 || k < 1 || k > m || k > 96) return TN_EINVAL;
    if (need(m, k) > (size_t)TN_NOALLOC_SCRATCH_DOUBLES) return TN_ESCRATCH;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double* base = nullptr;
    TN_TRY(scratch_address(&base));
    Arena ar;                                   // a view of the static array: no allocation
    ar.base = reinterpret_cast<char*>(base);
    ar.cap = sizeof(double) * (size_t)TN_NOALLOC_SCRATCH_DOUBLES;

    TsvdStats stats;
    int status = truncated_svd(st, ar, dM, m, k, dU, dS, dV, warm, &stats);
    if (status == TN_ENOMEM) return TN_ESCRATCH;
    if (status != TN_OK && status != TN_ENOCONV) return status;
    TN_CUDA(cudaStreamSynchronize(st));
    return status;
}
