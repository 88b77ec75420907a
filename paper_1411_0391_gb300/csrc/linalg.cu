// Small dense factorisations (one thread block per matrix) and the truncated
// SVD used for the CTMRG projectors.
//
// Truncated SVD of an m x m matrix M (top k triplets):
//   m <= SMALL_MAX: one-sided Jacobi SVD of M itself;
//   otherwise subspace iteration with kk = k + oversampling columns:
//     Y = orth(M Om), Z = orth(M^T Y), B = Y^T M Z = Ub Sb Vb^T (Jacobi),
//     repeated with Om = Z until the top-k Ritz values stop changing;
//     U = Y Ub, V = Z Vb.  orth() is the shifted Cholesky-QR3 of Fukaya et al.
//     (shifted CholQR, then CholQR twice): all products run as GEMMs over the
//     whole GPU, only the kk x kk Cholesky runs in one block.
// The sign rule (largest |entry| of each column of U positive) is applied to
// the final m-long vectors.
#include <algorithm>
#include <cmath>
#include "common.cuh"
#include "kernels.cuh"
#include "smallla.cuh"

namespace tn {

// ---------------------------------------------------------------------------
// batched small SVD
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) svd_small_kernel(const double* __restrict__ Ain, int m, int n,
        double* __restrict__ Uout, double* __restrict__ Sout, double* __restrict__ Vout, int max_sweeps)
{
    extern __shared__ double sm[];
    double* U = sm;                 // m*n column-major
    double* V = U + m * n;          // n*n column-major
    double* key = V + n * n;        // n
    __shared__ int flag;
    (void)max_sweeps;
    dev_svd(Ain + (size_t)blockIdx.x * m * n, m, n, U, Sout + (size_t)blockIdx.x * n, V, key, &flag);
    double* Uo = Uout + (size_t)blockIdx.x * m * n;
    double* Vo = Vout + (size_t)blockIdx.x * n * n;
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) Uo[e] = U[(e % n) * m + e / n];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Vo[e] = V[(e % n) * n + e / n];
}

static size_t svd_smem(int m, int n) { return sizeof(double) * ((size_t)m * n + (size_t)n * n + n) + 64; }

int svd_small(cudaStream_t st, const double* A, int m, int n, int batch, double* U, double* S, double* V)
{
    if (n < 1 || m < n || m > SMALL_MAX || batch < 1) return TN_EINVAL;
    size_t smem = svd_smem(m, n);
    static std::atomic<unsigned long long> attr{0};
    TN_CUDA(tn_smem_optin(svd_small_kernel, (int)svd_smem(SMALL_MAX, SMALL_MAX), attr));
    svd_small_kernel<<<batch, 512, smem, st>>>(A, m, n, U, S, V, 60);
    TN_LAUNCHED();
    return TN_OK;
}

// ---------------------------------------------------------------------------
// batched symmetric eigendecomposition, eigenvalues ascending, sign rule on
// the eigenvectors
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) eigh_small_kernel(const double* __restrict__ Ain, int n,
        double* __restrict__ Wout, double* __restrict__ Vout, int max_sweeps)
{
    extern __shared__ double sm[];
    double* A = sm;                   // n*n
    double* V = A + n * n;            // n*n column-major
    double* cs = V + n * n;           // 2*(n/2+1)
    int* pq = (int*)(cs + 2 * (n / 2 + 1));
    __shared__ double red[32];
    (void)max_sweeps;
    dev_eigh(Ain + (size_t)blockIdx.x * n * n, n, A, Wout + (size_t)blockIdx.x * n, V, cs, pq, red);
    double* Vo = Vout + (size_t)blockIdx.x * n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Vo[e] = V[(e % n) * n + e / n];
}

static size_t eigh_smem(int n) { return sizeof(double) * (2 * (size_t)n * n + 2 * (n / 2 + 1)) + sizeof(int) * 2 * (n / 2 + 1) + 64; }

int eigh_small(cudaStream_t st, const double* A, int n, int batch, double* W, double* V)
{
    if (n < 1 || n > SMALL_MAX || batch < 1) return TN_EINVAL;
    static std::atomic<unsigned long long> attr{0};
    TN_CUDA(tn_smem_optin(eigh_small_kernel, (int)eigh_smem(SMALL_MAX), attr));
    eigh_small_kernel<<<batch, 512, eigh_smem(n), st>>>(A, n, W, V, 60);
    TN_LAUNCHED();
    return TN_OK;
}

// ---------------------------------------------------------------------------
// Cholesky inverse for the orthonormalisation; shift = c_shift * u * tr(G)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) chol_inv_kernel(const double* __restrict__ Gin, int n,
        double c_shift, double* __restrict__ Xout)
{
    extern __shared__ double sm[];
    const int ld = n | 1;        // odd row stride (see blk_chol_inv)
    double* G = sm;              // n*ld
    double* X = G + n * ld;      // n*ld scratch
    int* dead = (int*)(X + n * ld);
    __shared__ double red[32];
    double tr = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        G[i * ld + j] = Gin[e];
        if (i == j) tr += Gin[e];
    }
    tr = block_sum(tr, red);
    const double shift = c_shift * 1.1102230246251565e-16 * tr;
    double dmax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) { G[i * ld + i] += shift; dmax = fmax(dmax, G[i * ld + i]); }
    __syncthreads();
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
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Xout[e] = G[(e / n) * ld + e % n];
}

static size_t chol_smem(int n) { return sizeof(double) * 2 * (size_t)n * (n | 1) + sizeof(int) * n + 64; }

int chol_inv(cudaStream_t st, const double* G, int n, double c_shift, double* X)
{
    if (n < 1 || n > SMALL_MAX) return TN_EINVAL;
    static std::atomic<unsigned long long> attr{0};
    TN_CUDA(tn_smem_optin(chol_inv_kernel, (int)chol_smem(SMALL_MAX), attr));
    chol_inv_kernel<<<1, 512, chol_smem(n), st>>>(G, n, c_shift, X);
    TN_LAUNCHED();
    return TN_OK;
}

// Sign rule on the columns of row-major U (rows x cols), flipping V too.
__global__ void sign_fix_cols_kernel(double* U, double* V, int rows, int vrows, int cols)
{
    const int j = blockIdx.x;
    __shared__ double red[32];
    __shared__ int firsts[32];
    double mx = 0.0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) mx = fmax(mx, fabs(U[(size_t)i * cols + j]));
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        red[0] = m;
    }
    __syncthreads();
    mx = red[0];
    if (mx == 0.0) return;
    const double thr = mx * (1.0 - 1e-10);
    int first = rows;
    for (int i = threadIdx.x; i < rows; i += blockDim.x)
        if (fabs(U[(size_t)i * cols + j]) >= thr) { first = i; break; }
    for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
    if ((threadIdx.x & 31) == 0) firsts[threadIdx.x >> 5] = first;
    __syncthreads();
    if (threadIdx.x == 0) {
        int f = rows;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) f = min(f, firsts[w]);
        firsts[0] = f;
    }
    __syncthreads();
    if (U[(size_t)firsts[0] * cols + j] >= 0.0) return;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) U[(size_t)i * cols + j] = -U[(size_t)i * cols + j];
    if (V) for (int i = threadIdx.x; i < vrows; i += blockDim.x) V[(size_t)i * cols + j] = -V[(size_t)i * cols + j];
}

int sign_fix_cols(cudaStream_t st, double* U, double* V, int rows, int vrows, int cols)
{
    if (cols <= 0) return TN_OK;
    sign_fix_cols_kernel<<<cols, 256, 0, st>>>(U, V, rows, vrows, cols);
    TN_LAUNCHED();
    return TN_OK;
}

// ---------------------------------------------------------------------------
// orthonormalisation of Y (rows x cols, row-major)
// ---------------------------------------------------------------------------
// orth: shifted CholeskyQR3 (Fukaya et al.): a shifted pass, then two plain ones.
int orth(cudaStream_t st, Arena& ar, double* Y, int rows, int cols)
{
    size_t mk = ar.mark();
    double* T = ar.take((size_t)rows * cols);
    if (!T) { ar.release(mk); return TN_ENOMEM; }
    int s = orth2(st, ar, Y, T, rows, cols, true);
    ar.release(mk);
    return s;
}

// orth2: columns scaled to unit norm, then Cholesky-QR passes: for an
// ill-conditioned basis (shifted) a shifted FP64 CholeskyQR, which brings the
// condition number down to about sqrt(u) kappa, one plain FP64 CholeskyQR,
// which leaves an orthogonality error of about u kappa(Q_1)^2, and two
// first-order FP64 corrections, each squaring that error (the last pass of the
// CholeskyQR3 of Fukaya et al. replaced by products and an O(n^2) kernel); for
// a basis that is already close to orthogonal up to column scales (the Ritz
// panels of the subspace iteration) two plain CholeskyQR passes.
// tmp: rows x cols of caller scratch.
int orth2(cudaStream_t st, Arena& ar, double* Y, double* tmp, int rows, int cols, bool shifted)
{
    size_t mk = ar.mark();
    double* G = ar.take((size_t)cols * cols);
    double* X = ar.take((size_t)cols * cols);
    if (!G || !X) { ar.release(mk); return TN_ENOMEM; }
    TN_TRY(normalize_cols(st, Y, rows, cols));
    const double c_first = 11.0 * ((double)rows * cols + (double)cols * (cols + 1));
    for (int pass = 0; pass < 2; ++pass) {
        TN_TRY(gemm_splitk(st, ar, true, false, cols, cols, rows, 1.0, Y, cols, Y, cols, 0.0, G, cols));
        TN_TRY(chol_inv(st, G, cols, (shifted && pass == 0) ? c_first : 0.0, X));
        TN_TRY(gemm(st, false, false, rows, cols, cols, 1.0, Y, cols, 0, X, cols, 0, 0.0, tmp, cols, 0, 1));
        TN_CUDA(cudaMemcpyAsync(Y, tmp, sizeof(double) * rows * cols, cudaMemcpyDeviceToDevice, st));
    }
    ar.release(mk);
    if (shifted) TN_TRY(orth_fixes(st, ar, Y, tmp, rows, cols, 2));
    return TN_OK;
}

// ---------------------------------------------------------------------------
// truncated SVD
// ---------------------------------------------------------------------------
// Top-k triplets of the m x m matrix M (row-major).  m <= SMALL_MAX: one-sided
// Jacobi on M.  Otherwise subspace iteration on kk = k + max(16, 3k/4) columns
// (at most 112; 112 for k = 64: on flat loop spectra the convergence factor per
// iteration, (s_{kk+1}/s_k)^2, needs the wide oversampling):
//   Y = orth(M Om), Z = orth(M^T Y), T = M Z, B = Y^T T = Ub Sb Vb^T,
//   Ritz vectors U_r = Y Ub, V_r = Z Vb; the next basis is Om = V_r, so B is
//   nearly diagonal from the second iteration on.  Stop when every kept Ritz
//   pair has || M v_i - s_i u_i || = || T vb_i - s_i u_i || <= tol s_1 (an
//   absolute test: directions at the noise floor pass it too; tol = 1e-13 in
//   FP64, looser when the products with M run on the tensor cores), cap 16.
// All products run as (split-K) GEMMs over the GPU.  The kk x kk
// factorisations run in one block each: on the first iteration in FP64, later
// in FP32 with FP64 refinement by products (orth_mixed, svd_mixed), falling
// back to the FP64 Jacobi SVD if the residual stops decreasing.  No heap
// allocation: host data lives on the stack.
int truncated_svd(cudaStream_t st, Arena& ar, const double* M, int m, int k,
                  double* U, double* S, double* V, const double* warm, TsvdStats* stats, int kind, double tol)
{
    if (k < 1 || k > m) return TN_EINVAL;
    size_t mk = ar.mark();
    if (m <= SMALL_MAX) {
        double* Uf = ar.take((size_t)m * m);
        double* Sf = ar.take(m);
        double* Vf = ar.take((size_t)m * m);
        if (!Uf || !Sf || !Vf) { ar.release(mk); return TN_ENOMEM; }
        TN_TRY(svd_small(st, M, m, m, 1, Uf, Sf, Vf));
        TN_CUDA(cudaMemcpy2DAsync(U, k * sizeof(double), Uf, m * sizeof(double), k * sizeof(double), m, cudaMemcpyDeviceToDevice, st));
        TN_CUDA(cudaMemcpy2DAsync(V, k * sizeof(double), Vf, m * sizeof(double), k * sizeof(double), m, cudaMemcpyDeviceToDevice, st));
        TN_CUDA(cudaMemcpyAsync(S, Sf, k * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (stats) { stats->iterations = 0; }
        ar.release(mk);
        return TN_OK;
    }
    const int kk = tsvd_columns(m, k);
    double* Om = ar.take((size_t)m * kk);
    double* Y = ar.take((size_t)m * kk);
    double* Z = ar.take((size_t)m * kk);
    double* T = ar.take((size_t)m * kk);
    double* TV = ar.take((size_t)m * k);
    double* Ur = ar.take((size_t)m * k);
    double* B = ar.take((size_t)kk * kk);
    double* Ub = ar.take((size_t)kk * kk);
    double* Vb = ar.take((size_t)kk * kk);
    double* Sb = ar.take(kk);
    double* rn = ar.take(kk);
    if (!Om || !Y || !Z || !T || !TV || !Ur || !B || !Ub || !Vb || !Sb || !rn) { ar.release(mk); return TN_ENOMEM; }
    // start: the warm right vectors (k columns) and fresh random oversampling columns
    TN_TRY(hash_fill(st, Om, (long long)m * kk, 0x5eed0000ull + (unsigned long long)m * 131 + k));
    if (warm)
        TN_CUDA(cudaMemcpy2DAsync(Om, kk * sizeof(double), warm, k * sizeof(double), k * sizeof(double), m,
                                  cudaMemcpyDeviceToDevice, st));
    double hs[SMALL_MAX], hr[SMALL_MAX];
    const int max_it = 16;
    int it = 0;
    bool conv = false;
    bool exact_rr = false;          // Rayleigh-Ritz SVD by FP64 Jacobi instead of FP32 + refinement
    double prev_worst = 0.0;
    for (it = 1; it <= max_it; ++it) {
        const bool first = (it == 1);
        if (kind >= 0) TN_TRY(gemm_tc(st, ar, kind, false, false, m, kk, m, 1.0, M, m, Om, kk, 0.0, Y, kk));
        else TN_TRY(gemm_splitk(st, ar, false, false, m, kk, m, 1.0, M, m, Om, kk, 0.0, Y, kk));
        // the first basis (random or warm + random) may be ill conditioned: FP64 shifted
        // CholeskyQR3; afterwards the panels are near orthogonal and FP32 whitening +
        // FP64 fixes suffice
        const bool fp64_orth = first;
        if (fp64_orth) TN_TRY(orth2(st, ar, Y, T, m, kk, true));
        else TN_TRY(orth_mixed(st, ar, Y, T, m, kk, 2));
        if (kind >= 0) TN_TRY(gemm_tc(st, ar, kind, true, false, m, kk, m, 1.0, M, m, Y, kk, 0.0, Z, kk));
        else TN_TRY(gemm_splitk(st, ar, true, false, m, kk, m, 1.0, M, m, Y, kk, 0.0, Z, kk));
        if (fp64_orth) TN_TRY(orth2(st, ar, Z, T, m, kk, true));
        else TN_TRY(orth_mixed(st, ar, Z, T, m, kk, 2));
        if (kind >= 0) TN_TRY(gemm_tc(st, ar, kind, false, false, m, kk, m, 1.0, M, m, Z, kk, 0.0, T, kk));
        else TN_TRY(gemm_splitk(st, ar, false, false, m, kk, m, 1.0, M, m, Z, kk, 0.0, T, kk));
        TN_TRY(gemm_splitk(st, ar, true, false, kk, kk, m, 1.0, Y, kk, T, kk, 0.0, B, kk));
        if (exact_rr) TN_TRY(svd_small(st, B, kk, kk, 1, Ub, Sb, Vb));
        else TN_TRY(svd_mixed(st, ar, B, kk, Ub, Sb, Vb, 2));
        TN_TRY(gemm(st, false, false, m, k, kk, 1.0, Y, kk, 0, Ub, kk, 0, 0.0, Ur, k, 0, 1));     // U_r
        TN_TRY(gemm(st, false, false, m, k, kk, 1.0, T, kk, 0, Vb, kk, 0, 0.0, TV, k, 0, 1));     // M V_r
        TN_TRY(residual_norms(st, TV, k, Ur, k, Sb, m, k, rn));
        TN_TRY(gemm(st, false, false, m, kk, kk, 1.0, Z, kk, 0, Vb, kk, 0, 0.0, Om, kk, 0, 1));   // V_r -> next basis
        TN_CUDA(cudaMemcpyAsync(hs, Sb, kk * sizeof(double), cudaMemcpyDeviceToHost, st));
        TN_CUDA(cudaMemcpyAsync(hr, rn, k * sizeof(double), cudaMemcpyDeviceToHost, st));
        TN_CUDA(cudaStreamSynchronize(st));
        double worst = 0.0;
        for (int i = 0; i < k; ++i) worst = std::max(worst, hr[i]);
        if (worst <= tol * std::max(hs[0], 1e-300)) { conv = true; break; }
        // a residual that stopped falling may be the FP32 Jacobi's unresolved
        // near-degenerate pairs: take the exact FP64 Ritz SVD from here on (a
        // residual that still falls, if slowly, is the subspace iteration's own
        // rate, which the FP64 Jacobi -- about 20 ms on one SM -- would not help)
        if (!first && worst > 0.9 * prev_worst) exact_rr = true;
        prev_worst = worst;
    }
    if (it > max_it) it = max_it;
    TN_CUDA(cudaMemcpyAsync(U, Ur, sizeof(double) * m * k, cudaMemcpyDeviceToDevice, st));
    TN_CUDA(cudaMemcpy2DAsync(V, k * sizeof(double), Om, kk * sizeof(double), k * sizeof(double), m, cudaMemcpyDeviceToDevice, st));
    TN_CUDA(cudaMemcpyAsync(S, Sb, k * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TN_TRY(sign_fix_cols(st, U, V, m, m, k));
    if (stats) stats->iterations = it;
    ar.release(mk);
    return conv ? TN_OK : TN_ENOCONV;
}

int tsvd_columns(int m, int k) { return std::min(m, std::min(SMALL_MAX, k + std::max(16, (3 * k) / 4))); }

}  // namespace tn
