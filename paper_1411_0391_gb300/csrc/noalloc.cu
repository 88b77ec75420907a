// Allocation-free variant of the truncated SVD (tn_truncated_svd_noalloc).
//
// Some callers cannot allocate device memory at the point where they need the
// projector SVD: a process whose device memory is entirely reserved by another
// allocator (a framework's caching pool), code where the implicit device-wide
// synchronisation of cudaMalloc/cudaFree is not acceptable, or a plugin that is
// not allowed to own device allocations and has no context workspace to lend.
// This entry point takes only the caller's input and output buffers; its
// scratch is the file-scope device array below, of a fixed, modest size
// (TN_NOALLOC_SCRATCH_DOUBLES doubles, 4 MiB), which every GPU that loads the
// library holds until the process exits.
//
// The algorithm is that of tn_truncated_svd (one-sided Jacobi for m <= 112,
// subspace iteration with Rayleigh-Ritz otherwise), run on the same kernels.
#include <algorithm>
#include <cmath>
#include "common.cuh"
#include "kernels.cuh"
#include "smallla.cuh"

#define TN_NOALLOC_SCRATCH_DOUBLES (1 << 19)

// Shared by every call on a device; nothing in it is assumed to start at zero
// (each call writes every scratch entry before reading it).
static __device__ __align__(256) double g_noalloc_scratch[TN_NOALLOC_SCRATCH_DOUBLES];

namespace tn {

namespace {

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the symbol is only a stand-in; kernels need the address returned by
// cudaGetSymbolAddress with the device current.
constexpr int MAX_DEVICES = 64;
double* g_scratch_addr[MAX_DEVICES] = {nullptr};

int scratch_address(double** out)
{
    int dev = 0;
    TN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return TN_EINVAL;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        TN_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return TN_OK;
}

// Doubles of scratch the call (m, k) needs; mirrors the carving below.
size_t need(int m, int k)
{
    auto al = [](size_t n) { return tn_align256(n * sizeof(double)) / sizeof(double); };
    if (m <= SMALL_MAX) return al((size_t)m * m) * 2 + al(m);
    const int kk = std::min(m, std::min(SMALL_MAX, k + std::max(8, k / 4)));
    size_t base = 4 * al((size_t)m * kk) + 3 * al((size_t)kk * kk) + al(kk);
    size_t orth_part = 2 * al((size_t)kk * kk) + al((size_t)m * kk);
    return base + orth_part;
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

    if (m <= SMALL_MAX) {
        double* Uf = ar.take((size_t)m * m);
        double* Sf = ar.take(m);
        double* Vf = ar.take((size_t)m * m);
        if (!Uf || !Sf || !Vf) return TN_ESCRATCH;
        TN_TRY(svd_small(st, dM, m, m, 1, Uf, Sf, Vf));
        TN_CUDA(cudaMemcpy2DAsync(dU, k * sizeof(double), Uf, m * sizeof(double), k * sizeof(double), m, cudaMemcpyDeviceToDevice, st));
        TN_CUDA(cudaMemcpy2DAsync(dV, k * sizeof(double), Vf, m * sizeof(double), k * sizeof(double), m, cudaMemcpyDeviceToDevice, st));
        TN_CUDA(cudaMemcpyAsync(dS, Sf, k * sizeof(double), cudaMemcpyDeviceToDevice, st));
        TN_CUDA(cudaStreamSynchronize(st));
        return TN_OK;
    }
    const int kk = std::min(m, std::min(SMALL_MAX, k + std::max(8, k / 4)));
    double* Om = ar.take((size_t)m * kk);
    double* Y = ar.take((size_t)m * kk);
    double* Z = ar.take((size_t)m * kk);
    double* T = ar.take((size_t)m * kk);
    double* B = ar.take((size_t)kk * kk);
    double* Ub = ar.take((size_t)kk * kk);
    double* Sb = ar.take(kk);
    double* Vb = ar.take((size_t)kk * kk);
    if (!Om || !Y || !Z || !T || !B || !Ub || !Sb || !Vb) return TN_ESCRATCH;
    TN_TRY(hash_fill(st, Om, (long long)m * kk, 0x5eed0000ull + (unsigned long long)m * 131 + k));
    if (warm)
        TN_CUDA(cudaMemcpy2DAsync(Om, kk * sizeof(double), warm, k * sizeof(double), k * sizeof(double), m, cudaMemcpyDeviceToDevice, st));
    double prev[SMALL_MAX], cur[SMALL_MAX];     // host stack, no heap
    for (int i = 0; i < kk; ++i) prev[i] = -1.0;
    const int max_it = 16;
    int it = 0;
    bool conv = false;
    for (; it < max_it; ++it) {
        TN_TRY(gemm(st, false, false, m, kk, m, 1.0, dM, m, 0, Om, kk, 0, 0.0, Y, kk, 0, 1));
        TN_TRY(orth(st, ar, Y, m, kk));
        TN_TRY(gemm(st, true, false, m, kk, m, 1.0, dM, m, 0, Y, kk, 0, 0.0, Z, kk, 0, 1));
        TN_TRY(orth(st, ar, Z, m, kk));
        TN_TRY(gemm(st, false, false, m, kk, m, 1.0, dM, m, 0, Z, kk, 0, 0.0, T, kk, 0, 1));
        TN_TRY(gemm(st, true, false, kk, kk, m, 1.0, Y, kk, 0, T, kk, 0, 0.0, B, kk, 0, 1));
        TN_TRY(svd_small(st, B, kk, kk, 1, Ub, Sb, Vb));
        TN_CUDA(cudaMemcpyAsync(cur, Sb, kk * sizeof(double), cudaMemcpyDeviceToHost, st));
        TN_CUDA(cudaStreamSynchronize(st));
        double dmax = 0.0;
        for (int i = 0; i < k; ++i) dmax = std::max(dmax, std::fabs(cur[i] - prev[i]));
        for (int i = 0; i < kk; ++i) prev[i] = cur[i];
        std::swap(Om, Z);
        if (it >= 1 && dmax <= 1e-14 * std::max(cur[0], 1e-300)) { ++it; conv = true; break; }
    }
    TN_TRY(gemm(st, false, false, m, k, kk, 1.0, Y, kk, 0, Ub, kk, 0, 0.0, dU, k, 0, 1));
    TN_TRY(gemm(st, false, false, m, k, kk, 1.0, Om, kk, 0, Vb, kk, 0, 0.0, dV, k, 0, 1));
    TN_CUDA(cudaMemcpyAsync(dS, Sb, k * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TN_TRY(sign_fix_cols(st, dU, dV, m, m, k));
    TN_CUDA(cudaStreamSynchronize(st));
    return conv ? TN_OK : TN_ENOCONV;
}
