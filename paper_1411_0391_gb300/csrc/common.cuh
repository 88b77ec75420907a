// Shared infrastructure of the tnite library: status handling, the device
// workspace arena and small tensor views.  All device memory of a context is
// carved from the caller's workspace; nothing here calls cudaMalloc.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstddef>
#include <cstring>
#include <vector>
#include <string>
#include "tnite.h"

#define TN_TRY(expr) do { int _s = (expr); if (_s != TN_OK && _s != TN_ENOCONV) return _s; } while (0)
#define TN_CUDA(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) { tn_last_cuda_error(_e); return TN_ECUDA; } } while (0)

void tn_last_cuda_error(cudaError_t e);
void tn_count_launch();
// after every kernel launch: count it and surface launch errors
#define TN_LAUNCHED() do { tn_count_launch(); TN_CUDA(cudaGetLastError()); } while (0)

// Opt `kernel` into `bytes` of dynamic shared memory on the current device.
// The attribute belongs to the device, so the record of where it has been set
// (`done`, bit d for device d < 64) is per device; devices >= 64 set it on every
// call.  Setting it twice is harmless, so racing threads need no lock.
template <typename K>
inline cudaError_t tn_smem_optin(K kernel, int bytes, std::atomic<unsigned long long>& done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// Counter-based uniform number in [-1, 1): splitmix64 of (seed, index).
__host__ __device__ inline double tn_hash_uniform(unsigned long long seed, long long i)
{
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static inline size_t tn_align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bump allocator over a caller-owned device buffer.  mark()/release() give
// stack-like scratch regions.
struct Arena {
    char*  base = nullptr;
    size_t cap = 0, off = 0, peak = 0;
    bool   counting = false;     // size-only pass: no base pointer
    double* take(size_t n_doubles) {
        size_t bytes = tn_align256(n_doubles * sizeof(double));
        size_t at = off;
        off += bytes;
        if (off > peak) peak = off;
        if (counting) return nullptr;
        if (off > cap) return nullptr;
        return reinterpret_cast<double*>(base + at);
    }
    size_t mark() const { return off; }
    void release(size_t m) { off = m; }
};

// A dense row-major tensor on the device (rank <= 8).
struct DT {
    double* p = nullptr;
    int rank = 0;
    int dim[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long size() const { long long s = 1; for (int i = 0; i < rank; ++i) s *= dim[i]; return s; }
};

static inline DT dt(double* p, std::initializer_list<int> dims) {
    DT t; t.p = p; t.rank = 0;
    for (int d : dims) t.dim[t.rank++] = d;
    return t;
}
