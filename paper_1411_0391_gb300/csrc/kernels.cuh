// Internal (non-exported) entry points of the tnite library.
#pragma once
#include "common.cuh"

namespace tn {

struct TsvdStats { int iterations = 0; };

// basic.cu
int gemm(cudaStream_t st, bool ta, bool tb, int m, int n, int k, double alpha,
         const double* A, int lda, long long sA, const double* B, int ldb, long long sB,
         double beta, double* C, int ldc, long long sC, int batch);
int gemm_splitk(cudaStream_t st, Arena& ar, bool ta, bool tb, int m, int n, int k, double alpha,
                const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc);
int normalize_cols(cudaStream_t st, double* Y, int rows, int cols);
int residual_norms(cudaStream_t st, const double* R, int ldr, const double* U, int ldu, const double* s,
                   int rows, int k, double* rn);
int permute(cudaStream_t st, const double* in, double* out, int rank, const int* dims, const int* perm);
int scale_rows(cudaStream_t st, double* C, int m, int n, int ldc, double s);
int normalize_maxabs(cudaStream_t st, double* x, long long n, int batch, long long stride);
int fill(cudaStream_t st, double* x, long long n, double v);
int hash_fill(cudaStream_t st, double* x, long long n, unsigned long long seed);
int axpby(cudaStream_t st, double* y, const double* x, long long n, double a, double b);
int dfma_probe(cudaStream_t st, int iters, double* flops);   // FP64 FMA rate probe (no sync)
void set_autotune(int on);                                   // DGEMM tile autotuner on/off
int autotune_entries();                                      // shapes tuned so far

// linalg.cu
int svd_small(cudaStream_t st, const double* A, int m, int n, int batch, double* U, double* S, double* V);
int eigh_small(cudaStream_t st, const double* A, int n, int batch, double* W, double* V);
int chol_inv(cudaStream_t st, const double* G, int n, double c_shift, double* X);
int sign_fix_cols(cudaStream_t st, double* U, double* V, int rows, int vrows, int cols);
int orth(cudaStream_t st, Arena& ar, double* Y, int rows, int cols);
int orth2(cudaStream_t st, Arena& ar, double* Y, double* tmp, int rows, int cols, bool shifted);
int tsvd_columns(int m, int k);
// mixed.cu: FP32 factorisations refined to FP64 by matrix products
int orth_mixed(cudaStream_t st, Arena& ar, double* Y, double* tmp, int rows, int cols, int fixes);
int orth_fixes(cudaStream_t st, Arena& ar, double* Y, double* tmp, int rows, int cols, int fixes);
int svd_mixed(cudaStream_t st, Arena& ar, const double* B, int n, double* U, double* S, double* V, int steps);

// kind: arithmetic of the products with M (see gemm_any); tol: Ritz residual
// stopping threshold relative to the largest singular value.
int truncated_svd(cudaStream_t st, Arena& ar, const double* M, int m, int k,
                  double* U, double* S, double* V, const double* warm, TsvdStats* stats,
                  int kind = -1, double tol = 1e-13);

// tc_gemm.cu: split-precision products on the tensor cores (kind 0 = TF32 x3,
// 1 = BF16 x3); tc_status reads and clears the device-side wait flag.
int tc_tile_n(int m, int n);
size_t gemm_tc_scratch_bytes(int kind, int m, int n, int k);
int gemm_tc(cudaStream_t st, Arena& ar, int kind, bool ta, bool tb, int m, int n, int k, double alpha,
            const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc);
int tc_status(cudaStream_t st, int* status);
// runs a kernel whose bounded wait on an mbarrier expires (nothing arrives on it);
// *status = the device-side wait flag afterwards (3 when the wait expired)
int wait_selftest(cudaStream_t st, int* status);
// C = alpha op(A) op(B) + beta C (no batch) in the contraction arithmetic
// `kind`: -1 = FP64 SIMT, 0 = TF32 x3 tensor cores, 1 = BF16 x3.
int gemm_any(cudaStream_t st, Arena& ar, int kind, bool ta, bool tb, int m, int n, int k, double alpha,
             const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc);

// contract.cu: C = alpha * A.B (+ beta C when no output permutation is needed),
// einsum-style labels "ab,bcm->acm" (no traces, no batch labels).
int contract(cudaStream_t st, Arena& ar, const char* spec, const DT& A, const DT& B, const DT& C,
             double alpha = 1.0, double beta = 0.0, int kind = -1);
// out = in with axes permuted by a label spec "abcd->cabd"
int permute_spec(cudaStream_t st, const char* spec, const DT& in, const DT& out);

}  // namespace tn
