// 1D iMPS with environment recycling (Sec. III and V): the canonical form of a
// one-site iMPS, the iMPO step with the optimal truncation through the
// canonical form, gauge fixing by local fidelity and the renormalised gate,
// for the transverse-field Ising chain.  This is the case the paper checks
// against the exact energy; the matrices are small (bond chi <= 16, the
// iMPO-applied tensor 2 chi <= 32), so every routine is one thread block with
// its operands in shared memory.
//
// Conventions: A[s][l][r] (d = 2), row-major; the iMPO g[s'][s][kl][kr]
// (kappa = 2), Theta[s'][(kl, l)][(kr, r)] kappa-major (Sec. V.A).
#include <algorithm>
#include <cmath>
#include "common.cuh"
#include "kernels.cuh"
#include "smallla.cuh"

namespace tn {

namespace {

constexpr int IMPS_MAXN = 32;          // largest bond of a canonicalised tensor (2 chi)
constexpr int IMPS_THREADS = 256;

// g[s'][s][kl][kr] = sum_t gF[s',t] w[kl,t] w[kr,t] gF[t,s], gF = exp(h tau X / 2),
// w[0,t] = sqrt(cosh tau), w[1,t] = sqrt(sinh tau) z_t  (Eq. iMPO1 with the SVD
// of the bond gate split symmetrically)
__device__ double impo_entry(double h, double tau, int sp, int s, int kl, int kr)
{
    const double ch = cosh(0.5 * h * tau), sh = sinh(0.5 * h * tau);
    const double w0 = sqrt(cosh(tau)), w1 = sqrt(sinh(tau));
    double acc = 0.0;
    for (int t = 0; t < 2; ++t) {
        const double gl = (sp == t) ? ch : sh, gr = (t == s) ? ch : sh;
        const double z = t == 0 ? 1.0 : -1.0;
        const double wl = kl == 0 ? w0 : w1 * z, wr = kr == 0 ? w0 : w1 * z;
        acc += gl * wl * wr * gr;
    }
    return acc;
}

// C (n x p) = A (n x m) B (m x p), all row-major in shared memory, block-wide
__device__ void sm_mm(const double* A, const double* B, double* C, int n, int m, int p)
{
    for (int e = threadIdx.x; e < n * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(A[i * m + k], B[k * p + j], acc);
        C[e] = acc;
    }
    __syncthreads();
}

__device__ double sm_norm(const double* x, int n, double* red)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fma(x[i], x[i], acc);
    return sqrt(block_sum(acc, red));
}

__device__ double sm_maxabs(const double* x, int n, double* red)
{
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(x[i]));
    m = warp_max(m);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
        red[0] = v;
    }
    __syncthreads();
    const double v = red[0];
    __syncthreads();
    return v;
}

// Eigen-square-root factors of a symmetric PSD V (n x n): with V = W diag(w) W^T
// (negative w clipped), F = diag(sqrt w) W^T and Finv = W diag(1/sqrt w) (zero
// below 1e-14 max w) -- the Y, Y^{-1} of step (i) -- or, transposed, X and X^{-1}.
// Eigenvectors come from dev_eigh as rows (Wr[i*n + j] = component j of vector i).
struct EigScratch { double* A; double* w; double* Wr; double* cs; int* pq; };

__device__ void sqrt_factors(const double* V, int n, EigScratch es, double* red, double* F, double* Finv,
                             bool transposed)
{
    dev_eigh(V, n, es.A, es.w, es.Wr, es.cs, es.pq, red);
    double wmax = 0.0;
    for (int k = 0; k < n; ++k) wmax = fmax(wmax, es.w[k]);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const double wi = fmax(es.w[i], 0.0), wj = fmax(es.w[j], 0.0);
        const double ri = sqrt(wi);
        const double inv_j = (wj >= 1e-14 * wmax && wj > 0.0) ? 1.0 / sqrt(wj) : 0.0;
        if (!transposed) {
            F[e] = ri * es.Wr[i * n + j];                 // Y = D^{1/2} W^T
            Finv[e] = es.Wr[j * n + i] * inv_j;           // Y^{-1} = W D^{-1/2}
        } else {
            const double rj = sqrt(wj);
            const double inv_i = (wi >= 1e-14 * wmax && wi > 0.0) ? 1.0 / ri : 0.0;
            F[e] = es.Wr[j * n + i] * rj;                 // X = W' D'^{1/2}
            Finv[e] = inv_i * es.Wr[i * n + j];           // X^{-1} = D'^{-1/2} W'^T
        }
    }
    __syncthreads();
}

struct CanonOut {
    double* G;       // d x n x n canonical Gamma
    double* lam;     // n
    double* ML;      // n x n left map (Gamma ~ ML A MR)
    double* MR;      // n x n right map
    double* Aw;      // d x n x n weighted sqrt(lam) Gamma sqrt(lam), unit norm (optional)
    int* iters;
};

// Canonical form of a one-site iMPS, Sec. III.A steps (i)-(iii), from Gamma = A,
// lambda uniform: V_L = sum_s (lam G^s)^T (lam G^s) = Y^T Y, V_R = sum_s (G^s lam)
// (G^s lam)^T = X X^T, Y lam X = U lam~ V^T, G~^s = V^T X^{-1} G^s Y^{-1} U; repeated
// until the n_watch largest weights change by less than tol lam_1.  One block.
__global__ void __launch_bounds__(IMPS_THREADS) imps_canon_kernel(const double* __restrict__ Ain, int n, double tol,
                                                                 int max_iter, int n_watch, CanonOut out)
{
    extern __shared__ double sm[];
    const int nn = n * n;
    double* G = sm;                  // 2 nn
    double* T = G + 2 * nn;          // 2 nn
    double* VL = T + 2 * nn;         // nn each below
    double* VR = VL + nn;
    double* Y = VR + nn;
    double* Yi = Y + nn;
    double* X = Yi + nn;
    double* Xi = X + nn;
    double* B = Xi + nn;
    double* U = B + nn;
    double* Vs = U + nn;
    double* left = Vs + nn;
    double* right = left + nn;
    double* ML = right + nn;
    double* MR = ML + nn;
    double* tmp = MR + nn;
    double* eA = tmp + nn;
    double* eW = eA + nn;
    double* ew = eW + nn;            // n
    double* lam = ew + n;            // n
    double* lamn = lam + n;          // n
    double* S = lamn + n;            // n
    double* key = S + n;             // n
    double* cs = key + n;            // 2 (n/2 + 1)
    int* pq = reinterpret_cast<int*>(cs + 2 * (n / 2 + 1));
    __shared__ double red[32];
    __shared__ int flag;
    __shared__ int done;
    EigScratch es{eA, ew, eW, cs, pq};

    for (int e = threadIdx.x; e < 2 * nn; e += blockDim.x) G[e] = Ain[e];
    for (int e = threadIdx.x; e < nn; e += blockDim.x) ML[e] = MR[e] = (e / n == e % n) ? 1.0 : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = 1.0 / sqrt((double)n);
    __syncthreads();
    const int watch = (n_watch > 0 && n_watch < n) ? n_watch : n;
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
        // V_L[r][q] = sum_{s,l} lam_l^2 G[s,l,r] G[s,l,q];  V_R[l][q] = sum_{s,r} lam_r^2 G[s,l,r] G[s,q,r]
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int a = e / n, b = e % n;
            double vl = 0.0, vr = 0.0;
            for (int s = 0; s < 2; ++s)
                for (int k = 0; k < n; ++k) {
                    const double l2 = lam[k] * lam[k];
                    vl = fma(l2 * G[s * nn + k * n + a], G[s * nn + k * n + b], vl);
                    vr = fma(l2 * G[s * nn + a * n + k], G[s * nn + b * n + k], vr);
                }
            VL[e] = vl;
            VR[e] = vr;
        }
        __syncthreads();
        sqrt_factors(VL, n, es, red, Y, Yi, false);
        sqrt_factors(VR, n, es, red, X, Xi, true);
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {        // B = Y diag(lam) X
            const int i = e / n, j = e % n;
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc = fma(Y[i * n + k] * lam[k], X[k * n + j], acc);
            B[e] = acc;
        }
        __syncthreads();
        dev_svd(B, n, n, U, S, Vs, key, &flag);                     // U, Vs column-major
        double nrm = 0.0;
        for (int k = 0; k < n; ++k) nrm += S[k] * S[k];
        nrm = sqrt(nrm);
        for (int k = threadIdx.x; k < n; k += blockDim.x) lamn[k] = nrm > 0.0 ? S[k] / nrm : S[k];
        // left = V^T X^{-1}, right = Y^{-1} U
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int i = e / n, j = e % n;
            double l = 0.0, r = 0.0;
            for (int k = 0; k < n; ++k) {
                l = fma(Vs[i * n + k], Xi[k * n + j], l);          // (V^T)[i][k] = V[k][i] = Vs[i*n + k]
                r = fma(Yi[i * n + k], U[j * n + k], r);           // U[k][j] = U[j*n + k]
            }
            left[e] = l;
            right[e] = r;
        }
        __syncthreads();
        // G <- left G^s right, unit norm
        for (int s = 0; s < 2; ++s) sm_mm(left, G + s * nn, T + s * nn, n, n, n);
        for (int s = 0; s < 2; ++s) sm_mm(T + s * nn, right, G + s * nn, n, n, n);
        const double gn = sm_norm(G, 2 * nn, red);
        for (int e = threadIdx.x; e < 2 * nn; e += blockDim.x) G[e] /= gn;
        // ML <- left ML, MR <- MR right, each divided by its largest |entry|
        sm_mm(left, ML, tmp, n, n, n);
        double m = sm_maxabs(tmp, nn, red);
        for (int e = threadIdx.x; e < nn; e += blockDim.x) ML[e] = m > 0.0 ? tmp[e] / m : tmp[e];
        __syncthreads();
        sm_mm(MR, right, tmp, n, n, n);
        m = sm_maxabs(tmp, nn, red);
        for (int e = threadIdx.x; e < nn; e += blockDim.x) MR[e] = m > 0.0 ? tmp[e] / m : tmp[e];
        __syncthreads();
        double d = 0.0;
        for (int k = 0; k < watch; ++k) d = fmax(d, fabs(lamn[k] - lam[k]));
        d = lamn[0] > 0.0 ? d / lamn[0] : d;
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) lam[k] = lamn[k];
        if (threadIdx.x == 0) done = d < tol ? 1 : 0;
        __syncthreads();
        if (done) break;
    }
    if (it > max_iter) it = max_iter;
    for (int e = threadIdx.x; e < 2 * nn; e += blockDim.x) out.G[e] = G[e];
    for (int e = threadIdx.x; e < nn; e += blockDim.x) { out.ML[e] = ML[e]; out.MR[e] = MR[e]; }
    for (int k = threadIdx.x; k < n; k += blockDim.x) out.lam[k] = lam[k];
    if (out.Aw) {                                           // sqrt(lam) G sqrt(lam), unit norm
        for (int e = threadIdx.x; e < 2 * nn; e += blockDim.x) {
            const int a = (e % nn) / n, b = e % n;
            T[e] = sqrt(lam[a]) * G[e] * sqrt(lam[b]);
        }
        __syncthreads();
        const double an = sm_norm(T, 2 * nn, red);
        for (int e = threadIdx.x; e < 2 * nn; e += blockDim.x) out.Aw[e] = T[e] / an;
    }
    if (threadIdx.x == 0 && out.iters) *out.iters = it;
}

size_t canon_smem(int n)
{
    return sizeof(double) * (4 * (size_t)n * n + 16 * (size_t)n * n + 6 * n + 2 * (n / 2 + 1)) +
           sizeof(int) * 2 * (n / 2 + 1) + 64;
}

// Theta[s'][(kl,l)][(kr,r)] = sum_s g[s'][s][kl][kr] A[s][l][r]   (chi -> 2 chi)
__global__ void imps_mpo_kernel(const double* __restrict__ A, int chi, double h, double tau, double* __restrict__ Th)
{
    const int n = 2 * chi, nn = n * n, cc = chi * chi;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * nn; e += gridDim.x * blockDim.x) {
        const int sp = e / nn, L = (e % nn) / n, R = e % n;
        const int kl = L / chi, l = L % chi, kr = R / chi, r = R % chi;
        Th[e] = impo_entry(h, tau, sp, 0, kl, kr) * A[l * chi + r] + impo_entry(h, tau, sp, 1, kl, kr) * A[cc + l * chi + r];
    }
}

// Truncation through the canonical form of Theta (n = 2 chi): Q = sqrt(lam_chi) ML[:chi, :]
// (chi x n), P = MR[:, :chi] sqrt(lam_chi) (n x chi), At^s = Q Theta^s P, unit norm.
__global__ void __launch_bounds__(IMPS_THREADS) imps_truncate_kernel(const double* __restrict__ Th, int chi,
        const double* __restrict__ lam, const double* __restrict__ ML, const double* __restrict__ MR,
        double* __restrict__ At, double* __restrict__ P, double* __restrict__ Q)
{
    extern __shared__ double sm[];
    const int n = 2 * chi;
    double* Qs = sm;                 // chi x n
    double* Ps = Qs + chi * n;       // n x chi
    double* T1 = Ps + n * chi;       // chi x n
    double* Ao = T1 + chi * n;       // 2 chi chi
    __shared__ double red[32];
    for (int e = threadIdx.x; e < chi * n; e += blockDim.x) {
        const int a = e / n, l = e % n;
        Qs[e] = sqrt(lam[a]) * ML[a * n + l];
        const int r = e / chi, b = e % chi;
        Ps[e] = MR[r * n + b] * sqrt(lam[b]);
    }
    __syncthreads();
    for (int s = 0; s < 2; ++s) {
        sm_mm(Qs, Th + s * n * n, T1, chi, n, n);
        sm_mm(T1, Ps, Ao + s * chi * chi, chi, n, chi);
    }
    const double an = sm_norm(Ao, 2 * chi * chi, red);
    for (int e = threadIdx.x; e < 2 * chi * chi; e += blockDim.x) At[e] = Ao[e] / an;
    for (int e = threadIdx.x; e < chi * n; e += blockDim.x) { P[e] = Ps[e]; Q[e] = Qs[e]; }
}

// Gauge fixing of Sec. III.B.2: U maximising F = sum_s Tr(U A^s U^T B^sT), by
// M = sum_s A^s U^T B^sT = W S V^T, U <- V W^T until U changes by less than tol.
// Start: the polar factor of the kappa = 0 leg map L0 = (sqrt(lam1) MLc) Q[:, :chi]
// (for small tau the kappa = 0 block of Theta = g A_0 is A_0 up to a factor, so
// B ~ L0 A_0 (...)); the iteration only climbs to the nearest local maximum, and
// from the identity it can stop in one that depends on the canonical forms'
// sign conventions.
__global__ void __launch_bounds__(IMPS_THREADS) imps_gauge_kernel(const double* __restrict__ A,
        const double* __restrict__ Bt, int chi, const double* __restrict__ lam1, const double* __restrict__ MLc,
        const double* __restrict__ Q, double tol, int max_iter, double* __restrict__ Uout, double* __restrict__ F)
{
    extern __shared__ double sm[];
    const int cc = chi * chi;
    double* Us = sm;               // cc
    double* M = Us + cc;
    double* T1 = M + cc;
    double* Wm = T1 + cc;          // column-major SVD factors
    double* Vm = Wm + cc;
    double* Sv = Vm + cc;          // chi
    double* key = Sv + chi;        // chi
    __shared__ double red[32];
    __shared__ int flag;
    __shared__ int stop;
    {
        const int n = 2 * chi;
        for (int e = threadIdx.x; e < cc; e += blockDim.x) {      // L0[i][j], j < chi (kappa = 0 columns)
            const int i = e / chi, j = e % chi;
            double acc = 0.0;
            for (int k = 0; k < chi; ++k) acc = fma(MLc[i * chi + k], Q[k * n + j], acc);
            T1[e] = sqrt(lam1[i]) * acc;
        }
        __syncthreads();
        dev_svd(T1, chi, chi, Wm, Sv, Vm, key, &flag);             // L0 = W S V^T, column-major factors
        for (int e = threadIdx.x; e < cc; e += blockDim.x) {      // U = W V^T
            const int i = e / chi, j = e % chi;
            double acc = 0.0;
            for (int k = 0; k < chi; ++k) acc = fma(Wm[k * chi + i], Vm[k * chi + j], acc);
            Us[e] = acc;
        }
        __syncthreads();
    }
    for (int it = 0; it < max_iter; ++it) {
        // M[a][d] = sum_s sum_{b,c} A[s,a,b] U[c,b] B[s,d,c]
        for (int e = threadIdx.x; e < cc; e += blockDim.x) {       // T1[a][c] = sum_s... staged per s below
            M[e] = 0.0;
        }
        __syncthreads();
        for (int s = 0; s < 2; ++s) {
            for (int e = threadIdx.x; e < cc; e += blockDim.x) {   // T1[a][c] = sum_b A[s,a,b] U[c,b]
                const int a = e / chi, c = e % chi;
                double acc = 0.0;
                for (int b = 0; b < chi; ++b) acc = fma(A[s * cc + a * chi + b], Us[c * chi + b], acc);
                T1[e] = acc;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < cc; e += blockDim.x) {   // M[a][d] += sum_c T1[a][c] B[s,d,c]
                const int a = e / chi, d = e % chi;
                double acc = 0.0;
                for (int c = 0; c < chi; ++c) acc = fma(T1[a * chi + c], Bt[s * cc + d * chi + c], acc);
                M[e] += acc;
            }
            __syncthreads();
        }
        dev_svd(M, chi, chi, Wm, Sv, Vm, key, &flag);
        double change = 0.0;
        for (int e = 0; e < cc; ++e) {                             // U = V W^T (every thread)
            const int i = e / chi, j = e % chi;
            double acc = 0.0;
            for (int k = 0; k < chi; ++k) acc = fma(Vm[k * chi + i], Wm[k * chi + j], acc);
            change = fmax(change, fabs(acc - Us[e]));
        }
        __syncthreads();
        for (int e = threadIdx.x; e < cc; e += blockDim.x) {
            const int i = e / chi, j = e % chi;
            double acc = 0.0;
            for (int k = 0; k < chi; ++k) acc = fma(Vm[k * chi + i], Wm[k * chi + j], acc);
            Us[e] = acc;
        }
        if (threadIdx.x == 0) stop = change < tol ? 1 : 0;
        __syncthreads();
        if (stop) break;
    }
    // F = sum_s sum U[a,b] A[s,b,c] U[d,c] B[s,a,d]
    double part = 0.0;
    for (int s = 0; s < 2; ++s)
        for (int e = threadIdx.x; e < cc; e += blockDim.x) {
            const int a = e / chi, d = e % chi;
            double acc = 0.0;
            for (int b = 0; b < chi; ++b)
                for (int c = 0; c < chi; ++c) acc += Us[a * chi + b] * A[s * cc + b * chi + c] * Us[d * chi + c];
            part += acc * Bt[s * cc + a * chi + d];
        }
    const double f = block_sum(part, red);
    for (int e = threadIdx.x; e < cc; e += blockDim.x) Uout[e] = Us[e];
    if (threadIdx.x == 0) *F = f;
}

// Renormalised gate of Sec. V.B: KL = U^T (sqrt(lam1) MLc) Q (chi x 2chi),
// KR = P (MRc sqrt(lam1)) U (2chi x chi).
__global__ void __launch_bounds__(IMPS_THREADS) imps_gate_kernel(const double* __restrict__ U, const double* __restrict__ lam1,
        const double* __restrict__ MLc, const double* __restrict__ MRc, const double* __restrict__ P,
        const double* __restrict__ Q, int chi, double* __restrict__ KL, double* __restrict__ KR)
{
    extern __shared__ double sm[];
    const int n = 2 * chi, cc = chi * chi;
    double* T1 = sm;               // cc
    double* T2 = T1 + cc;          // cc
    double* Us = T2 + cc;          // cc
    for (int e = threadIdx.x; e < cc; e += blockDim.x) Us[e] = U[e];
    // T1 = U^T (sqrt(lam1) MLc);  T2 = (MRc sqrt(lam1)) U
    for (int e = threadIdx.x; e < cc; e += blockDim.x) {
        const int i = e / chi, j = e % chi;
        double a = 0.0, b = 0.0;
        for (int k = 0; k < chi; ++k) {
            a = fma(U[k * chi + i], sqrt(lam1[k]) * MLc[k * chi + j], a);
            b = fma(MRc[i * chi + k] * sqrt(lam1[k]), U[k * chi + j], b);
        }
        T1[e] = a;
        T2[e] = b;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < chi * n; e += blockDim.x) {      // KL = T1 Q
        const int i = e / n, j = e % n;
        double acc = 0.0;
        for (int k = 0; k < chi; ++k) acc = fma(T1[i * chi + k], Q[k * n + j], acc);
        KL[e] = acc;
    }
    for (int e = threadIdx.x; e < n * chi; e += blockDim.x) {      // KR = P T2
        const int i = e / chi, j = e % chi;
        double acc = 0.0;
        for (int k = 0; k < chi; ++k) acc = fma(P[i * chi + k], T2[k * chi + j], acc);
        KR[e] = acc;
    }
}

// One recycled step: A <- KL (g A)^s KR, unit norm.
__global__ void __launch_bounds__(IMPS_THREADS) imps_recycled_step_kernel(double* __restrict__ A, int chi, double h,
        double tau, const double* __restrict__ KL, const double* __restrict__ KR)
{
    extern __shared__ double sm[];
    const int n = 2 * chi, cc = chi * chi;
    double* Th = sm;                // 2 n n
    double* T1 = Th + 2 * n * n;    // chi n
    double* Ao = T1 + chi * n;      // 2 cc
    __shared__ double red[32];
    for (int e = threadIdx.x; e < 2 * n * n; e += blockDim.x) {
        const int sp = e / (n * n), L = (e % (n * n)) / n, R = e % n;
        const int kl = L / chi, l = L % chi, kr = R / chi, r = R % chi;
        Th[e] = impo_entry(h, tau, sp, 0, kl, kr) * A[l * chi + r] + impo_entry(h, tau, sp, 1, kl, kr) * A[cc + l * chi + r];
    }
    __syncthreads();
    for (int s = 0; s < 2; ++s) {
        sm_mm(KL, Th + s * n * n, T1, chi, n, n);
        sm_mm(T1, KR, Ao + s * cc, chi, n, chi);
    }
    const double an = sm_norm(Ao, 2 * cc, red);
    for (int e = threadIdx.x; e < 2 * cc; e += blockDim.x) A[e] = Ao[e] / an;
}

// <ZZ>, <X>, e = -<ZZ> - h <X> from the canonical form (Gamma, lam): the
// environments of lam Gamma lam Gamma lam are identities.
__global__ void __launch_bounds__(IMPS_THREADS) imps_observables_kernel(const double* __restrict__ G,
        const double* __restrict__ lam, int chi, double h, double* __restrict__ out)
{
    extern __shared__ double sm[];
    const int cc = chi * chi;
    double* T2 = sm;               // [s][t][a][c]: 4 cc
    double* th = T2 + 4 * cc;      // [s][a][b]: 2 cc
    __shared__ double r1[4];
    __shared__ double r2[16];
    __shared__ double red[32];
    for (int e = threadIdx.x; e < 2 * cc; e += blockDim.x) {
        const int a = (e % cc) / chi, b = e % chi;
        th[e] = lam[a] * G[e] * lam[b];
    }
    for (int e = threadIdx.x; e < 4 * cc; e += blockDim.x) {
        const int st = e / cc, a = (e % cc) / chi, c = e % chi;
        const int s = st >> 1, t = st & 1;
        double acc = 0.0;
        for (int b = 0; b < chi; ++b) acc = fma(G[s * cc + a * chi + b] * lam[b], G[t * cc + b * chi + c], acc);
        T2[e] = lam[a] * acc * lam[c];
    }
    __syncthreads();
    for (int q = 0; q < 16; ++q) {                 // rho2[(s t)][(u v)] = sum_{a,c} T2[st][a][c] T2[uv][a][c]
        const int st = q / 4, uv = q % 4;
        double part = 0.0;
        for (int e = threadIdx.x; e < cc; e += blockDim.x) part = fma(T2[st * cc + e], T2[uv * cc + e], part);
        const double v = block_sum(part, red);
        if (threadIdx.x == 0) r2[q] = v;
    }
    for (int q = 0; q < 4; ++q) {                  // rho1[s][t] = sum_{a,b} th[s,a,b] th[t,a,b]
        const int s = q / 2, t = q % 2;
        double part = 0.0;
        for (int e = threadIdx.x; e < cc; e += blockDim.x) part = fma(th[s * cc + e], th[t * cc + e], part);
        const double v = block_sum(part, red);
        if (threadIdx.x == 0) r1[q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr2 = 0.0, zz = 0.0;
        for (int st = 0; st < 4; ++st) {
            const double v = r2[st * 4 + st];
            tr2 += v;
            zz += (((st >> 1) == (st & 1)) ? 1.0 : -1.0) * v;
        }
        zz /= tr2;
        const double x = (r1[1] + r1[2]) / (r1[0] + r1[3]);
        out[0] = zz;
        out[1] = x;
        out[2] = -zz - h * x;
    }
}

// Buffers of the recycling and plain steps, carved from the caller's workspace.
struct ImpsBufs {
    double *Th, *G, *lam, *ML, *MR, *A0, *At, *P, *Q, *G1, *lam1, *MLc, *MRc, *A1, *U, *KL, *KR, *F, *obs;
    int* iters;
};

bool carve(Arena& ar, int chi, ImpsBufs& b)
{
    const size_t n = 2 * (size_t)chi, c = chi;
    b.Th = ar.take(2 * n * n); b.G = ar.take(2 * n * n); b.lam = ar.take(n); b.ML = ar.take(n * n); b.MR = ar.take(n * n);
    b.A0 = ar.take(2 * c * c); b.At = ar.take(2 * c * c); b.P = ar.take(n * c); b.Q = ar.take(c * n);
    b.G1 = ar.take(2 * c * c); b.lam1 = ar.take(c); b.MLc = ar.take(c * c); b.MRc = ar.take(c * c);
    b.A1 = ar.take(2 * c * c); b.U = ar.take(c * c); b.KL = ar.take(c * n); b.KR = ar.take(n * c);
    b.F = ar.take(8); b.obs = ar.take(8);
    b.iters = reinterpret_cast<int*>(ar.take(8));
    return b.Th && b.G && b.lam && b.ML && b.MR && b.A0 && b.At && b.P && b.Q && b.G1 && b.lam1 && b.MLc && b.MRc &&
           b.A1 && b.U && b.KL && b.KR && b.F && b.obs && b.iters;
}

size_t imps_bytes(int chi)
{
    Arena ar;
    ar.counting = true;
    ImpsBufs b;
    carve(ar, chi, b);
    return ar.peak + 256;
}

int launch_canon(cudaStream_t st, const double* A, int n, double tol, int max_iter, int n_watch, CanonOut o)
{
    static std::atomic<unsigned long long> attr{0};
    TN_CUDA(tn_smem_optin(imps_canon_kernel, (int)canon_smem(IMPS_MAXN), attr));
    imps_canon_kernel<<<1, IMPS_THREADS, canon_smem(n), st>>>(A, n, tol, max_iter, n_watch, o);
    TN_LAUNCHED();
    return TN_OK;
}

// One plain step: A <- truncate(g A); keeps Theta's canonical data and P, Q in b.
int plain_step(cudaStream_t st, ImpsBufs& b, double* A, int chi, double h, double tau)
{
    const int n = 2 * chi;
    imps_mpo_kernel<<<8, 256, 0, st>>>(A, chi, h, tau, b.Th);
    TN_LAUNCHED();
    CanonOut o{b.G, b.lam, b.ML, b.MR, nullptr, b.iters};
    TN_TRY(launch_canon(st, b.Th, n, 1e-12, 2000, chi, o));     // kept weights only (reading of Sec. V)
    const size_t smem = sizeof(double) * (3 * (size_t)chi * n + 2 * (size_t)chi * chi);
    imps_truncate_kernel<<<1, IMPS_THREADS, smem, st>>>(b.Th, chi, b.lam, b.ML, b.MR, b.At, b.P, b.Q);
    TN_LAUNCHED();
    return TN_OK;
}

}  // namespace

}  // namespace tn

using namespace tn;

extern "C" {

size_t tn_imps_workspace_bytes(int chi)
{
    if (chi < 1 || 2 * chi > IMPS_MAXN) return 0;
    return imps_bytes(chi);
}

static int imps_args(const double* dA, int chi, double tau, void* work, size_t bytes, Arena& ar, ImpsBufs& b)
{
    if (!dA || !work || chi < 1 || 2 * chi > IMPS_MAXN || !(tau > 0.0) || !std::isfinite(tau)) return TN_EINVAL;
    if (bytes < imps_bytes(chi)) return TN_ENOMEM;
    const uintptr_t base = (reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255);
    ar.base = reinterpret_cast<char*>(base);
    ar.cap = bytes - (base - reinterpret_cast<uintptr_t>(work));
    return carve(ar, chi, b) ? TN_OK : TN_ENOMEM;
}

int tn_imps_itebd(double* dA, int chi, double h, double tau, int n_steps, void* work, size_t bytes, void* stream)
{
    Arena ar;
    ImpsBufs b;
    if (n_steps < 0 || !std::isfinite(h)) return TN_EINVAL;
    TN_TRY(imps_args(dA, chi, tau, work, bytes, ar, b));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < n_steps; ++i) {
        TN_TRY(plain_step(st, b, dA, chi, h, tau));
        TN_CUDA(cudaMemcpyAsync(dA, b.At, sizeof(double) * 2 * chi * chi, cudaMemcpyDeviceToDevice, st));
    }
    TN_CUDA(cudaStreamSynchronize(st));
    return TN_OK;
}

int tn_imps_recycle(double* dA, int chi, double h, double tau, int n_re, double* fidelity, void* work, size_t bytes,
                    void* stream)
{
    Arena ar;
    ImpsBufs b;
    if (n_re < 1 || !std::isfinite(h)) return TN_EINVAL;
    TN_TRY(imps_args(dA, chi, tau, work, bytes, ar, b));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t cc = (size_t)chi * chi;
    // A_0: weighted canonical form of A
    CanonOut o0{b.G1, b.lam1, b.MLc, b.MRc, b.A0, b.iters};
    TN_TRY(launch_canon(st, dA, chi, 1e-13, 2000, 0, o0));
    // the plain step from A_0 (Theta, its canonical truncation, P, Q)
    TN_TRY(plain_step(st, b, b.A0, chi, h, tau));
    // canonical form of A~: A~_1 = Q_c A~ P_c with the maps MLc, MRc and weights lam1
    CanonOut o1{b.G1, b.lam1, b.MLc, b.MRc, b.A1, b.iters};
    TN_TRY(launch_canon(st, b.At, chi, 1e-13, 2000, 0, o1));
    // gauge fix A~_1 ~ U A_0 U^T
    const size_t gsm = sizeof(double) * (5 * cc + 2 * chi);
    imps_gauge_kernel<<<1, IMPS_THREADS, gsm, st>>>(b.A0, b.A1, chi, b.lam1, b.MLc, b.Q, 1e-12, 2000, b.U, b.F);
    TN_LAUNCHED();
    imps_gate_kernel<<<1, IMPS_THREADS, sizeof(double) * 3 * cc, st>>>(b.U, b.lam1, b.MLc, b.MRc, b.P, b.Q, chi,
                                                                      b.KL, b.KR);
    TN_LAUNCHED();
    TN_CUDA(cudaMemcpyAsync(dA, b.A0, sizeof(double) * 2 * cc, cudaMemcpyDeviceToDevice, st));
    const int n = 2 * chi;
    const size_t rsm = sizeof(double) * (2 * (size_t)n * n + (size_t)chi * n + 2 * cc);
    for (int k = 0; k < n_re; ++k) {
        imps_recycled_step_kernel<<<1, IMPS_THREADS, rsm, st>>>(dA, chi, h, tau, b.KL, b.KR);
        TN_LAUNCHED();
    }
    double F = 0.0;
    TN_CUDA(cudaMemcpyAsync(&F, b.F, sizeof(double), cudaMemcpyDeviceToHost, st));
    TN_CUDA(cudaStreamSynchronize(st));
    if (fidelity) *fidelity = F;
    return std::isfinite(F) ? TN_OK : TN_ENUMERIC;
}

int tn_imps_observables(const double* dA, int chi, double h, double* out, void* work, size_t bytes, void* stream)
{
    Arena ar;
    ImpsBufs b;
    if (!out || !std::isfinite(h)) return TN_EINVAL;
    TN_TRY(imps_args(dA, chi, 1.0, work, bytes, ar, b));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CanonOut o{b.G1, b.lam1, b.MLc, b.MRc, nullptr, b.iters};
    TN_TRY(launch_canon(st, dA, chi, 1e-13, 2000, 0, o));
    imps_observables_kernel<<<1, IMPS_THREADS, sizeof(double) * 6 * (size_t)chi * chi, st>>>(b.G1, b.lam1, chi, h,
                                                                                           b.obs);
    TN_LAUNCHED();
    TN_CUDA(cudaMemcpyAsync(out, b.obs, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    TN_CUDA(cudaStreamSynchronize(st));
    return TN_OK;
}

}  // extern "C"
