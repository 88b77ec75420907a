// Mixed-precision small dense factorisations for the projector SVD.
//
// GB300 runs FP64 at about two fused multiply-adds per clock per SM, FP32 at
// 128: a factorisation that lives on one SM (a Cholesky or a Jacobi sweep of
// a 112 x 112 matrix) is 64 times cheaper in FP32.  The factorisations here
// are therefore done in FP32 and brought to FP64 accuracy by refinement steps
// that are plain FP64 matrix products, which run over the whole GPU.
//
//   orth_mixed    columns of a tall Y made orthonormal: FP32 Cholesky of the
//                 scaled Gram matrix (whitening), then first-order FP64
//                 corrections Y <- Y (I - F), F = striu(E) + diag(E)/2 for
//                 Y^T Y = I + E, each squaring the orthogonality error; a
//                 correction whose E is not small falls back to the FP64
//                 Cholesky inverse in the same kernel.
//   svd_mixed     SVD of a small square B: one-sided (Hestenes) Jacobi in
//                 FP32, then the refinement of Ogita and Aishima (JSIAM
//                 Letters / Japan J. Indust. Appl. Math., iterative refinement
//                 for the singular value decomposition based on matrix
//                 multiplication): with R = I - U^T U, S = I - V^T V and
//                 T = U^T B V, the corrections U <- U (I + F), V <- V (I + G)
//                 solve, to first order, F + F^T = R, G + G^T = S and
//                 T + F^T Sigma + Sigma G diagonal; pairs whose correction
//                 would not be small (clusters) are only re-orthogonalised.
#include <algorithm>
#include <cmath>
#include "common.cuh"
#include "kernels.cuh"
#include "smallla.cuh"

namespace tn {

namespace {

__device__ __forceinline__ float warp_sum_f(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// whitening: X = D^{-1/2} R^{-1} with R^T R the FP32 Cholesky of D^{-1/2} G D^{-1/2}
// (D = diag G).  Pivots at the FP32 noise floor mark a column dead (zero in X).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) chol32_whiten_kernel(const double* __restrict__ G, int n, float shift,
                                                            double* __restrict__ X)
{
    extern __shared__ float fs[];
    const int ld = n | 1;          // odd row stride (see blk_chol_inv)
    float* R = fs;                 // n*ld: the scaled Gram matrix, then R^{-1}
    float* Ri = R + n * ld;        // n*ld scratch
    __shared__ double dsc[SMALL_MAX];
    __shared__ int dead[SMALL_MAX];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = G[(size_t)i * n + i];
        dsc[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        R[i * ld + j] = (float)(G[e] * dsc[i] * dsc[j]) + (i == j ? shift : 0.0f);
    }
    __syncthreads();
    const float thr = 1e-5f;       // a unit diagonal carries FP32 rounding of ~n * 6e-8
    blk_chol_inv<float>(R, n, ld, thr, Ri, dead);   // Ri: scratch; R^{-1} lands in R
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, c = e % n;
        X[e] = dead[c] ? 0.0 : dsc[i] * (double)R[i * ld + c];
    }
}

// First-order orthogonality correction from G = Y^T Y: X = I - F with
// F = striu(E) + diag(E)/2, E = G - I, when max |E| <= 1/32 (the error after
// the step is O(E^2)); otherwise the FP64 Cholesky inverse of G (CholeskyQR).
// Dead columns (G_jj = 0) stay zero.  The first-order case is elementwise and
// spread over the blocks (each block finds max |E| itself, reading G from L2);
// the Cholesky fallback runs in block 0 alone.
constexpr int FIX_BLOCKS = 28;
__global__ void __launch_bounds__(256) orth_fix_kernel(const double* __restrict__ Gin, int n, double* __restrict__ Xo)
{
    extern __shared__ double ds[];
    const int ld = n | 1;          // odd row stride (see blk_chol_inv)
    __shared__ double red[32];
    double emax = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const bool zero_col = Gin[(size_t)i * n + i] == 0.0 || Gin[(size_t)j * n + j] == 0.0;
        if (!zero_col) emax = fmax(emax, fabs(Gin[e] - (i == j ? 1.0 : 0.0)));
    }
    emax = warp_max(emax);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        red[0] = m;
    }
    __syncthreads();
    emax = red[0];
    __syncthreads();
    if (emax <= 1.0 / 32.0) {
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
            const int i = e / n, j = e % n;
            const double g = Gin[e];
            double x;
            if (Gin[(size_t)j * n + j] == 0.0) x = 0.0;
            else if (i == j) x = 1.0 - 0.5 * (g - 1.0);
            else x = i < j ? -g : 0.0;
            Xo[e] = x;
        }
        return;
    }
    if (blockIdx.x != 0) return;
    double* G = ds;                // n*ld
    double* X = G + n * ld;        // n*ld
    int* dead = reinterpret_cast<int*>(X + n * ld);
    double dmax = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        G[i * ld + j] = Gin[e];
        if (i == j) dmax = fmax(dmax, Gin[e]);
    }
    dmax = warp_max(dmax);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        red[0] = m;
    }
    __syncthreads();
    blk_chol_inv<double>(G, n, ld, 1e-26 * red[0], X, dead);     // X: scratch; the inverse lands in G
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Xo[e] = G[(e / n) * ld + e % n];
}

size_t chol32_smem(int n) { return sizeof(float) * 2 * (size_t)n * (n | 1) + 64; }
size_t orthfix_smem(int n) { return sizeof(double) * 2 * (size_t)n * (n | 1) + sizeof(int) * n + 64; }

// ---------------------------------------------------------------------------
// FP32 one-sided Jacobi SVD of B (n x n row-major FP64) -> U0, V0 (n x n
// row-major FP64, columns sorted by descending singular value; columns of
// zero norm give zero U columns).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float half_sum_f(float v, unsigned mask)
{
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, 16);
    return v;
}

// One pair per half-warp (16 lanes): with 1024 threads every pair of a round
// (n/2 <= 56) runs at once, so a round costs one pair's latency.
__global__ void __launch_bounds__(1024) svd32_kernel(const double* __restrict__ B, int n,
                                                     double* __restrict__ U0, double* __restrict__ V0)
{
    extern __shared__ float fs[];
    float* A = fs;                 // column-major n x n: column j at A + j*n
    float* V = A + n * n;          // column-major n x n
    __shared__ float nrm[SMALL_MAX];
    __shared__ int rank[SMALL_MAX];
    __shared__ double red[32];
    __shared__ int rotated;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double mx = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) mx = fmax(mx, fabs(B[e]));
    mx = warp_max(mx);
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < nw; ++w) m = fmax(m, red[w]);
        red[0] = m > 0.0 ? 1.0 / m : 0.0;
    }
    __syncthreads();
    const double sc = red[0];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        A[j * n + i] = (float)(B[e] * sc);
        V[j * n + i] = i == j ? 1.0f : 0.0f;
    }
    __syncthreads();
    const float tol = fmaxf(1e-6f, 2.0f * n * 6e-8f);
    const int M = n + (n & 1);
    const int hw = threadIdx.x >> 4, hl = threadIdx.x & 15, nhw = blockDim.x >> 4;
    const unsigned hmask = 0xffffu << (16 * ((threadIdx.x >> 4) & 1));
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < M - 1; ++r) {
            for (int k = hw; k < M / 2; k += nhw) {
                int p, q;
                rr_pair(M, r, k, p, q);
                if (q >= n) continue;              // uniform over the half-warp
                float* ap = A + p * n;
                float* aq = A + q * n;
                float al = 0.0f, be = 0.0f, ga = 0.0f;
                for (int i = hl; i < n; i += 16) {
                    const float x = ap[i], y = aq[i];
                    al = fmaf(x, x, al); be = fmaf(y, y, be); ga = fmaf(x, y, ga);
                }
                al = half_sum_f(al, hmask); be = half_sum_f(be, hmask); ga = half_sum_f(ga, hmask);
                // sqrt(al) sqrt(be), not sqrt(al be): on the graded Ritz blocks of a loop matrix
                // (column norms from 1 down to 1e-15 and below) the product underflows in FP32,
                // the test never passes and every sweep rotates again up to the sweep cap
                if (ga == 0.0f || fabsf(ga) <= tol * sqrtf(al) * sqrtf(be) || al < 1e-30f || be < 1e-30f) continue;
                const float zeta = (be - al) / (2.0f * ga);
                const float az = fabsf(zeta);      // zeta^2 overflows FP32 beyond 1.8e19: t = 1 / (2 |zeta|) there
                const float t = (zeta >= 0.0f ? 1.0f : -1.0f) / (az + (az > 1e18f ? az : sqrtf(1.0f + az * az)));
                const float c = rsqrtf(1.0f + t * t), s = c * t;
                for (int i = hl; i < n; i += 16) {
                    const float x = ap[i], y = aq[i];
                    ap[i] = c * x - s * y; aq[i] = s * x + c * y;
                }
                float* vp = V + p * n;
                float* vq = V + q * n;
                for (int i = hl; i < n; i += 16) {
                    const float x = vp[i], y = vq[i];
                    vp[i] = c * x - s * y; vq[i] = s * x + c * y;
                }
                if (hl == 0) rotated = 1;
            }
            __syncthreads();
        }
        if (!rotated) break;
    }
    for (int j = warp; j < n; j += nw) {
        float acc = 0.0f;
        for (int i = lane; i < n; i += 32) acc = fmaf(A[j * n + i], A[j * n + i], acc);
        acc = warp_sum_f(acc);
        if (lane == 0) nrm[j] = sqrtf(acc);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        int rk = 0;
        for (int i = 0; i < n; ++i) rk += (nrm[i] > nrm[j]) || (nrm[i] == nrm[j] && i < j);
        rank[j] = rk;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;          // row i, source column j
        const float s = nrm[j];
        U0[(size_t)i * n + rank[j]] = s > 0.0f ? (double)A[j * n + i] / (double)s : 0.0;
        V0[(size_t)i * n + rank[j]] = (double)V[j * n + i];
    }
}

// One Ogita-Aishima step: from Rm = U^T U, Sm = V^T V, T = U^T B V (n x n,
// row-major) produce the corrections F, G (U <- U + U F, V <- V + V G) and the
// refined singular values S.  Elementwise, with two FP64 divisions per entry:
// spread over OA_BLOCKS blocks (on one SM the divisions alone take ~0.1 ms at
// n = 112); every block recomputes the n refined values it needs.
constexpr int OA_THREADS = 256;
constexpr int OA_BLOCKS = 49;          // 112^2 / 256 entries: one per thread
__global__ void __launch_bounds__(OA_THREADS) oa_step_kernel(const double* __restrict__ Rm, const double* __restrict__ Sm,
                                                             const double* __restrict__ T, int n, double* __restrict__ F,
                                                             double* __restrict__ G, double* __restrict__ S)
{
    __shared__ double sig[SMALL_MAX];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double rii = 1.0 - Rm[(size_t)i * n + i], sii = 1.0 - Sm[(size_t)i * n + i];
        const double den = 1.0 - 0.5 * (rii + sii);
        sig[i] = den > 0.0 ? T[(size_t)i * n + i] / den : 0.0;
        if (blockIdx.x == 0) S[i] = sig[i];
    }
    __syncthreads();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int i = e / n, j = e % n;
        const double r = (i == j ? 1.0 : 0.0) - Rm[e];
        const double s = (i == j ? 1.0 : 0.0) - Sm[e];
        double f = 0.5 * r, g = 0.5 * s;
        if (i != j) {
            const double si = sig[i], sj = sig[j];
            const double a = -T[e] - sj * r;
            const double b = -T[(size_t)j * n + i] - sj * s;
            const double den = si * si - sj * sj;
            if (den != 0.0) {
                const double fc = (sj * a + si * b) / den;
                const double gc = (si * a + sj * b) / den;
                if (fabs(fc) <= 0.125 && fabs(gc) <= 0.125) { f = fc; g = gc; }   // else: a cluster pair
            }
        }
        F[e] = f;
        G[e] = g;
    }
}

size_t svd32_smem(int n) { return sizeof(float) * 2 * (size_t)n * n + 64; }

}  // namespace

// Y (rows x cols, row-major) to orthonormal columns spanning the same space
// (up to dead directions): FP32 whitening, then `fixes` FP64 correction steps.
int orth_mixed(cudaStream_t st, Arena& ar, double* Y, double* tmp, int rows, int cols, int fixes)
{
    if (cols < 1 || cols > SMALL_MAX) return TN_EINVAL;
    static std::atomic<unsigned long long> attr0{0};
    static std::atomic<unsigned long long> attr1{0};
    TN_CUDA(tn_smem_optin(chol32_whiten_kernel, (int)chol32_smem(SMALL_MAX), attr0));
    TN_CUDA(tn_smem_optin(orth_fix_kernel, (int)orthfix_smem(SMALL_MAX), attr1));
    size_t mk = ar.mark();
    double* G = ar.take((size_t)cols * cols);
    double* X = ar.take((size_t)cols * cols);
    if (!G || !X) { ar.release(mk); return TN_ENOMEM; }
    for (int pass = 0; pass <= fixes; ++pass) {
        TN_TRY(gemm_splitk(st, ar, true, false, cols, cols, rows, 1.0, Y, cols, Y, cols, 0.0, G, cols));
        if (pass == 0) chol32_whiten_kernel<<<1, 256, chol32_smem(cols), st>>>(G, cols, 0.0f, X);
        else orth_fix_kernel<<<FIX_BLOCKS, 256, orthfix_smem(cols), st>>>(G, cols, X);
        TN_LAUNCHED();
        TN_TRY(gemm(st, false, false, rows, cols, cols, 1.0, Y, cols, 0, X, cols, 0, 0.0, tmp, cols, 0, 1));
        TN_CUDA(cudaMemcpyAsync(Y, tmp, sizeof(double) * rows * cols, cudaMemcpyDeviceToDevice, st));
    }
    ar.release(mk);
    return TN_OK;
}

// `fixes` first-order FP64 orthogonality corrections of Y (rows x cols), for a
// basis already close to orthonormal (each squares the error; the kernel falls
// back to the FP64 Cholesky inverse where the error is not small).
int orth_fixes(cudaStream_t st, Arena& ar, double* Y, double* tmp, int rows, int cols, int fixes)
{
    if (cols < 1 || cols > SMALL_MAX) return TN_EINVAL;
    static std::atomic<unsigned long long> attr{0};
    TN_CUDA(tn_smem_optin(orth_fix_kernel, (int)orthfix_smem(SMALL_MAX), attr));
    size_t mk = ar.mark();
    double* G = ar.take((size_t)cols * cols);
    double* X = ar.take((size_t)cols * cols);
    if (!G || !X) { ar.release(mk); return TN_ENOMEM; }
    for (int pass = 0; pass < fixes; ++pass) {
        TN_TRY(gemm_splitk(st, ar, true, false, cols, cols, rows, 1.0, Y, cols, Y, cols, 0.0, G, cols));
        orth_fix_kernel<<<FIX_BLOCKS, 256, orthfix_smem(cols), st>>>(G, cols, X);
        TN_LAUNCHED();
        TN_TRY(gemm(st, false, false, rows, cols, cols, 1.0, Y, cols, 0, X, cols, 0, 0.0, tmp, cols, 0, 1));
        TN_CUDA(cudaMemcpyAsync(Y, tmp, sizeof(double) * rows * cols, cudaMemcpyDeviceToDevice, st));
    }
    ar.release(mk);
    return TN_OK;
}

// SVD of the n x n row-major B: U, V (n x n row-major, columns = singular
// vectors, descending), S (n).  FP32 Jacobi, then `steps` FP64 refinement steps.
int svd_mixed(cudaStream_t st, Arena& ar, const double* B, int n, double* U, double* S, double* V, int steps)
{
    if (n < 1 || n > SMALL_MAX) return TN_EINVAL;
    static std::atomic<unsigned long long> attr{0};
    TN_CUDA(tn_smem_optin(svd32_kernel, (int)svd32_smem(SMALL_MAX), attr));
    size_t mk = ar.mark();
    const size_t nn = (size_t)n * n;
    double* Rm = ar.take(nn);
    double* Sm = ar.take(nn);
    double* BV = ar.take(nn);
    double* T = ar.take(nn);
    double* F = ar.take(nn);
    double* G = ar.take(nn);
    if (!Rm || !Sm || !BV || !T || !F || !G) { ar.release(mk); return TN_ENOMEM; }
    svd32_kernel<<<1, 1024, svd32_smem(n), st>>>(B, n, U, V);
    TN_LAUNCHED();
    for (int it = 0; it < steps; ++it) {
        TN_TRY(gemm(st, true, false, n, n, n, 1.0, U, n, 0, U, n, 0, 0.0, Rm, n, 0, 1));
        TN_TRY(gemm(st, true, false, n, n, n, 1.0, V, n, 0, V, n, 0, 0.0, Sm, n, 0, 1));
        TN_TRY(gemm(st, false, false, n, n, n, 1.0, B, n, 0, V, n, 0, 0.0, BV, n, 0, 1));
        TN_TRY(gemm(st, true, false, n, n, n, 1.0, U, n, 0, BV, n, 0, 0.0, T, n, 0, 1));
        oa_step_kernel<<<OA_BLOCKS, OA_THREADS, 0, st>>>(Rm, Sm, T, n, F, G, S);
        TN_LAUNCHED();
        // U <- U + U F, V <- V + V G (BV and Rm are free again: staging copies)
        TN_CUDA(cudaMemcpyAsync(BV, U, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
        TN_TRY(gemm(st, false, false, n, n, n, 1.0, BV, n, 0, F, n, 0, 1.0, U, n, 0, 1));
        TN_CUDA(cudaMemcpyAsync(Rm, V, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
        TN_TRY(gemm(st, false, false, n, n, n, 1.0, Rm, n, 0, G, n, 0, 1.0, V, n, 0, 1));
    }
    if (steps == 0) {     // singular values of the FP32 factorisation: diag(U^T B V)
        TN_TRY(gemm(st, false, false, n, n, n, 1.0, B, n, 0, V, n, 0, 0.0, BV, n, 0, 1));
        TN_TRY(gemm(st, true, false, n, n, n, 1.0, U, n, 0, BV, n, 0, 0.0, T, n, 0, 1));
        TN_CUDA(cudaMemcpy2DAsync(S, sizeof(double), T, sizeof(double) * (n + 1), sizeof(double), n,
                                  cudaMemcpyDeviceToDevice, st));
    }
    ar.release(mk);
    return TN_OK;
}

}  // namespace tn
