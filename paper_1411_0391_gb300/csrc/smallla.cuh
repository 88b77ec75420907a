// Block-level dense linear algebra on shared-memory matrices, in double.
//
// One thread block owns one matrix.  GB300 issues FP64 at a low rate per SM,
// so these routines are meant for the small (<= 112) matrices of the method:
// Rayleigh-Ritz problems of the projector SVD, corner spectra, bond-matrix
// SVDs, Gram matrices.  Pairs of indices are rotated in parallel in the
// round-robin (circle) order: in every round each index appears in exactly one
// pair, so the rotations of a round touch disjoint rows/columns.
#pragma once
#include <cuda_runtime.h>

namespace tn {

constexpr int SMALL_MAX = 112;

__device__ __forceinline__ void rr_pair(int M, int r, int k, int& p, int& q)
{
    if (k == 0) { p = r; q = M - 1; }
    else { p = (r + k) % (M - 1); q = (r - k + (M - 1)) % (M - 1); }
    if (p > q) { int t = p; p = q; q = t; }
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum; red must hold 32 doubles; every thread gets the result.
__device__ __forceinline__ double block_sum(double v, double* red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (w == 0) { t = warp_sum(t); if (lane == 0) red[0] = t; }
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}

// One-sided (Hestenes) Jacobi SVD.  A: column-major m x n (column j at A + j*m),
// n <= m, overwritten by U*S (columns orthogonal); V: column-major n x n,
// set to the accumulated rotations.  Returns the number of sweeps.
static __device__ int blk_svd_onesided(double* A, int m, int n, double* V, int* flag, int max_sweeps)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = (e % n == e / n) ? 1.0 : 0.0;
    const int M = n + (n & 1);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) *flag = 0;
        __syncthreads();
        for (int r = 0; r < M - 1; ++r) {
            for (int k = warp; k < M / 2; k += nw) {
                int p, q;
                rr_pair(M, r, k, p, q);
                if (q >= n) continue;
                double* ap = A + (size_t)p * m;
                double* aq = A + (size_t)q * m;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = lane; i < m; i += 32) {
                    double x = ap[i], y = aq[i];
                    al = fma(x, x, al); be = fma(y, y, be); ga = fma(x, y, ga);
                }
                al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
                if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al) * sqrt(be)) continue;   // no underflow of al be
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = lane; i < m; i += 32) {
                    double x = ap[i], y = aq[i];
                    ap[i] = c * x - s * y; aq[i] = s * x + c * y;
                }
                double* vp = V + (size_t)p * n;
                double* vq = V + (size_t)q * n;
                for (int i = lane; i < n; i += 32) {
                    double x = vp[i], y = vq[i];
                    vp[i] = c * x - s * y; vq[i] = s * x + c * y;
                }
                if (lane == 0) *flag = 1;
            }
            __syncthreads();
        }
        if (*flag == 0) break;
        __syncthreads();
    }
    __syncthreads();
    return sweep;
}

// Two-sided cyclic Jacobi eigendecomposition of a symmetric matrix.
// A: row-major n x n (symmetric), overwritten (its diagonal ends as the
// eigenvalues); V: column-major n x n eigenvectors.  cs: 2*(n/2+1) doubles,
// pq: 2*(n/2+1) ints of scratch.
static __device__ int blk_eigh_jacobi(double* A, int n, double* V, double* cs, int* pq, double* red, int max_sweeps)
{
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = (e % n == e / n) ? 1.0 : 0.0;
    __syncthreads();
    const int M = n + (n & 1), H = M / 2;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            double v = A[e];
            if (e % n == e / n) dia += v * v; else off += v * v;
        }
        off = block_sum(off, red);
        dia = block_sum(dia, red);
        // relative off-diagonal norm at the rounding floor of n-term sums
        const double eps_n = fmax(1e-15, (double)n * 1e-16);
        if (off <= eps_n * eps_n * (dia + off) || off == 0.0) break;
        for (int r = 0; r < M - 1; ++r) {
            for (int k = threadIdx.x; k < H; k += blockDim.x) {
                int p, q;
                rr_pair(M, r, k, p, q);
                double c = 1.0, s = 0.0;
                if (q < n) {
                    double apq = A[p * n + q];
                    if (fabs(apq) > 1e-300) {
                        double th = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                        double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + hypot(1.0, th));
                        c = 1.0 / sqrt(1.0 + t * t); s = t * c;
                    }
                } else { q = p; }
                cs[2 * k] = c; cs[2 * k + 1] = s; pq[2 * k] = p; pq[2 * k + 1] = q;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < H * n; e += blockDim.x) {      // rows
                int k = e / n, j = e % n;
                int p = pq[2 * k], q = pq[2 * k + 1];
                if (p == q) continue;
                double c = cs[2 * k], s = cs[2 * k + 1];
                double x = A[p * n + j], y = A[q * n + j];
                A[p * n + j] = c * x - s * y; A[q * n + j] = s * x + c * y;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < H * n; e += blockDim.x) {      // columns and V
                int k = e / n, j = e % n;
                int p = pq[2 * k], q = pq[2 * k + 1];
                if (p == q) continue;
                double c = cs[2 * k], s = cs[2 * k + 1];
                double x = A[j * n + p], y = A[j * n + q];
                A[j * n + p] = c * x - s * y; A[j * n + q] = s * x + c * y;
                double vx = V[p * n + j], vy = V[q * n + j];
                V[p * n + j] = c * vx - s * vy; V[q * n + j] = s * vx + c * vy;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    return sweep;
}

// Sign rule: for each column j (column-major n_rows x n_cols in U), find the
// largest |entry|; the first row within a relative 1e-10 of it decides the
// sign; a negative sign flips column j of U and of V (n_v rows).
static __device__ void blk_sign_fix(double* U, int n_rows, int n_cols, double* V, int n_v)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < n_cols; j += nw) {
        double* u = U + (size_t)j * n_rows;
        double mx = 0.0;
        for (int i = lane; i < n_rows; i += 32) mx = fmax(mx, fabs(u[i]));
        mx = warp_max(mx);
        if (mx == 0.0) continue;
        double thr = mx * (1.0 - 1e-10);
        int first = n_rows;
        for (int i = lane; i < n_rows; i += 32)
            if (fabs(u[i]) >= thr) { first = i; break; }
        for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
        bool neg = u[first] < 0.0;
        if (neg) {
            for (int i = lane; i < n_rows; i += 32) u[i] = -u[i];
            if (V) for (int i = lane; i < n_v; i += 32) V[(size_t)j * n_v + i] = -V[(size_t)j * n_v + i];
        }
    }
    __syncthreads();
}

// Cholesky G + shift I = R^T R (R upper) followed by X = R^{-1}.  G: row-major
// n x n, destroyed.  Pivots below dead_rel * max diagonal mark a column as
// linearly dependent: its column of X is zero (the orthonormalised basis then
// has a zero column there).  X: row-major n x n.
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Cholesky G = L L^T of the symmetric n x n matrix in shared memory (row-major,
// leading dimension ld, which callers make odd, n + 1 for even n: threads of a
// warp walk different rows, and an even row stride would put them on one
// shared-memory bank), then X = (L^T)^{-1} = R^{-1} (upper triangular), written
// over G.  Blocked in panels of CB = 16 columns so that the whole factorisation
// and inversion take a few dozen block barriers (n = 112: 7 panels), not a few
// per column -- on one SM the barriers, not the arithmetic, set the time:
//   panel p: warp 0 factors the panel's columns (rows p.. n-1) with
//            warp-synchronous steps; then every thread applies the rank-CB
//            update to the trailing lower triangle (rows and columns >= p + CB);
//   inverse: M = L^{-1} by block rows: the diagonal blocks' inverses (one warp
//            per block, forward substitution), then for block row I the blocks
//            J < I as M_IJ = -M_II sum_{K=J}^{I-1} L_IK M_KJ (two phases);
//   X = M^T.
// A pivot not above thr marks its column dead: L's column is zero below a unit
// diagonal and X's column is zero.  M: n x ld shared scratch; dead: n ints.
constexpr int CB = 16;

template <typename T>
__device__ void blk_chol_inv(T* G, int n, int ld, T thr, T* M, int* dead)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nthr = blockDim.x;
    for (int p = 0; p < n; p += CB) {
        const int pe = min(p + CB, n);
        if (warp == 0) {
            // unblocked Cholesky of columns p .. pe-1 over rows p .. n-1 (earlier panels'
            // contributions are already subtracted by their trailing updates)
            for (int j = p; j < pe; ++j) {
                T d = G[j * ld + j];
                for (int k = p; k < j; ++k) d -= G[j * ld + k] * G[j * ld + k];
                const bool isdead = !(d > thr);
                const T r = isdead ? T(1) : sqrt(d);
                for (int i = j + 1 + lane; i < n; i += 32) {
                    T v = G[i * ld + j];
                    for (int k = p; k < j; ++k) v -= G[i * ld + k] * G[j * ld + k];
                    G[i * ld + j] = isdead ? T(0) : v / r;
                }
                __syncwarp();
                if (lane == 0) { G[j * ld + j] = r; dead[j] = isdead ? 1 : 0; }
                __syncwarp();
            }
        }
        __syncthreads();
        // trailing update of the lower triangle: G[i][c] -= sum_{k in panel} L[i][k] L[c][k]
        const int m = n - pe;
        for (int e = threadIdx.x; e < m * m; e += nthr) {
            const int i = pe + e / m, c = pe + e % m;
            if (c > i) continue;
            T acc = G[i * ld + c];
            for (int k = p; k < pe; ++k) acc -= G[i * ld + k] * G[c * ld + k];
            G[i * ld + c] = acc;
        }
        __syncthreads();
    }
    // M = L^{-1}: diagonal blocks first (one warp each), then block rows
    const int nb = (n + CB - 1) / CB;
    const int nw = nthr >> 5;
    for (int I = warp; I < nb; I += nw) {
        const int p = I * CB, pe = min(p + CB, n);
        for (int c = p + lane; c < pe; c += 32) {          // column c of the block's inverse
            for (int i = p; i < pe; ++i) {
                T acc = (i == c) ? T(1) : T(0);
                if (i < c) { M[i * ld + c] = T(0); continue; }
                for (int l = c; l < i; ++l) acc -= G[i * ld + l] * M[l * ld + c];
                M[i * ld + c] = acc / G[i * ld + i];
            }
        }
    }
    __syncthreads();
    for (int I = 1; I < nb; ++I) {
        const int p = I * CB, pe = min(p + CB, n);
        // phase 1: T_IJ = sum_{K=J}^{I-1} L_IK M_KJ for every J < I, kept in M's upper triangle
        // (M_IJ itself is written in phase 2; the upper triangle of M is free)
        for (int e = threadIdx.x; e < (pe - p) * p; e += nthr) {
            const int i = p + e / p, c = e % p;             // row i of block row I, column c < p
            T acc = T(0);
            for (int l = c; l < p; ++l) acc += G[i * ld + l] * M[l * ld + c];
            M[c * ld + i] = acc;                              // transposed slot (c < p <= i): upper triangle
        }
        __syncthreads();
        // phase 2: M_IJ = -M_II T_IJ
        for (int e = threadIdx.x; e < (pe - p) * p; e += nthr) {
            const int i = p + e / p, c = e % p;
            T acc = T(0);
            for (int l = p; l <= i; ++l) acc += M[i * ld + l] * M[c * ld + l];
            M[i * ld + c] = -acc;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += nthr) {
        const int i = e / n, c = e % n;
        G[i * ld + c] = (i <= c && !dead[c]) ? M[c * ld + i] : T(0);
    }
    __syncthreads();
}

}  // namespace tn

namespace tn {

// Swap columns a and b of a column-major rows x cols matrix (block-wide).
__device__ __forceinline__ void blk_swap_cols(double* M, int rows, int a, int b)
{
    if (a == b) return;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        double t = M[(size_t)a * rows + i];
        M[(size_t)a * rows + i] = M[(size_t)b * rows + i];
        M[(size_t)b * rows + i] = t;
    }
}

// Full SVD of a row-major m x n matrix (n <= m) at Ain (any memory space).
// U: column-major m x n, V: column-major n x n, S: n, descending, sign rule
// applied.  key: n doubles of scratch.  flag: one int of shared scratch.
static __device__ void dev_svd(const double* Ain, int m, int n, double* U, double* S, double* V, double* key, int* flag)
{
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) U[(e % n) * m + e / n] = Ain[e];
    __syncthreads();
    blk_svd_onesided(U, m, n, V, flag, 60);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < n; j += nw) {
        double acc = 0.0;
        for (int i = lane; i < m; i += 32) acc = fma(U[j * m + i], U[j * m + i], acc);
        acc = warp_sum(acc);
        if (lane == 0) key[j] = sqrt(acc);
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {                   // selection sort by column swaps
        __shared__ int best;
        if (threadIdx.x == 0) {
            int b = j;
            for (int l = j + 1; l < n; ++l) if (key[l] > key[b]) b = l;
            best = b;
        }
        __syncthreads();
        int b = best;
        if (b != j) {
            blk_swap_cols(U, m, j, b);
            blk_swap_cols(V, n, j, b);
            __syncthreads();
            if (threadIdx.x == 0) { double t = key[j]; key[j] = key[b]; key[b] = t; }
        }
        __syncthreads();
    }
    for (int j = warp; j < n; j += nw) {
        double inv = key[j] > 0.0 ? 1.0 / key[j] : 0.0;
        for (int i = lane; i < m; i += 32) U[j * m + i] *= inv;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) S[j] = key[j];
    __syncthreads();
    blk_sign_fix(U, m, n, V, n);
}

// Symmetric eigendecomposition of a row-major n x n matrix at Ain (symmetrised
// on load): W ascending, V column-major eigenvectors with the sign rule.
// A: n*n scratch, cs: 2*(n/2+1) doubles, pq: 2*(n/2+1) ints, red: 32 doubles.
static __device__ void dev_eigh(const double* Ain, int n, double* A, double* W, double* V, double* cs, int* pq, double* red)
{
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        A[e] = 0.5 * (Ain[i * n + j] + Ain[j * n + i]);
    }
    __syncthreads();
    blk_eigh_jacobi(A, n, V, cs, pq, red, 60);
    for (int j = threadIdx.x; j < n; j += blockDim.x) W[j] = A[j * n + j];
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        __shared__ int best;
        if (threadIdx.x == 0) {
            int b = j;
            for (int l = j + 1; l < n; ++l) if (W[l] < W[b]) b = l;
            best = b;
        }
        __syncthreads();
        int b = best;
        if (b != j) {
            blk_swap_cols(V, n, j, b);
            __syncthreads();
            if (threadIdx.x == 0) { double t = W[j]; W[j] = W[b]; W[b] = t; }
        }
        __syncthreads();
    }
    blk_sign_fix(V, n, n, nullptr, 0);
}

}  // namespace tn
