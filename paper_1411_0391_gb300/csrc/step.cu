// One imaginary-time step of the full update with environment recycling:
// rows a1 (iPEPO), a2 (double layer), a7 (pre-truncation), a8 (bond
// environment), a9 (ALS), a10 (assembly), a11 (canonical form), a12 (gauge
// fixing), a13 (renormalised gate) and a14 (observables).
//
// The small iterative FP64 solvers (canonical form, pre-truncation, PSD
// projection, ALS, gauge fixing) each run as one thread block per link or per
// cell with all operands in shared memory; the contractions with the chi-sized
// environment run as GEMMs through the contraction planner.
#include <algorithm>
#include <cmath>
#include "ctx.cuh"
#include "smallla.cuh"

namespace tn {

// ============================================================================
// a1: iPEPO g[s'][s][l][r][d][u] = sum_t gF[s',t] w[l,t] w[r,t] w[d,t] w[u,t] gF[t,s]
//     gF = exp(h tau X / 2);  w[0,t] = sqrt(cosh(J tau)), w[1,t] = sqrt(sinh(J tau)) z_t
// ============================================================================
__global__ void pepo_kernel(double* g, double J, double h, double tau)
{
    const double ch = cosh(0.5 * h * tau), sh = sinh(0.5 * h * tau);
    const double gf[2][2] = {{ch, sh}, {sh, ch}};
    const double w0 = sqrt(cosh(J * tau)), w1 = sqrt(sinh(J * tau));
    const double w[2][2] = {{w0, w0}, {w1, -w1}};
    for (int e = threadIdx.x; e < 64; e += blockDim.x) {
        int u = e & 1, d = (e >> 1) & 1, r = (e >> 2) & 1, l = (e >> 3) & 1, s = (e >> 4) & 1, sp = (e >> 5) & 1;
        double acc = 0.0;
        for (int t = 0; t < 2; ++t) acc += gf[sp][t] * w[l][t] * w[r][t] * w[d][t] * w[u][t] * gf[t][s];
        g[e] = acc;
    }
}

int build_pepo(Ctx& c)
{
    pepo_kernel<<<1, 64, 0, c.st>>>(c.g, c.J, c.h, c.tau);
    TN_LAUNCHED();
    c.have_pepo = true;
    return TN_OK;
}

// Theta[s'][(kl,l)][(kr,r)][(kd,d)][(ku,u)] = sum_s g[s'][s][kl][kr][kd][ku] A[s][l][r][d][u]
__global__ void apply_pepo_kernel(const double* __restrict__ g, const double* __restrict__ A,
                                  double* __restrict__ T, int D)
{
    const int kD = 2 * D;
    const long long total = 2LL * kD * kD * kD * kD;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long r = e;
        int U = r % kD; r /= kD; int Dd = r % kD; r /= kD; int R = r % kD; r /= kD; int L = r % kD; r /= kD;
        int sp = (int)r;
        int kl = L / D, il = L % D, kr = R / D, ir = R % D, kd = Dd / D, id = Dd % D, ku = U / D, iu = U % D;
        int gi = ((kl * 2 + kr) * 2 + kd) * 2 + ku;
        long long ai = (((long long)il * D + ir) * D + id) * D + iu;
        const long long sA = (long long)D * D * D * D;
        T[e] = g[(sp * 2 + 0) * 16 + gi] * A[ai] + g[(sp * 2 + 1) * 16 + gi] * A[sA + ai];
    }
}

static int apply_pepo(Ctx& c, const double* A, double* T)
{
    const long long total = 2LL * c.kD * c.kD * c.kD * c.kD;
    int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 4);
    apply_pepo_kernel<<<blocks, 256, 0, c.st>>>(c.g, A, T, c.D);
    TN_LAUNCHED();
    return TN_OK;
}

// ============================================================================
// a2: double layer a[(l l')][(r r')][(d d')][(u u')] = sum_s A[s..] A[s..']
// ============================================================================
__global__ void double_layer_kernel(const double* __restrict__ A, double* __restrict__ a, int D)
{
    const int L = D * D;
    const long long total = (long long)L * L * L * L;
    const long long sA = (long long)D * D * D * D;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long r = e;
        int u = r % L; r /= L; int d = r % L; r /= L; int rr = r % L; r /= L; int l = (int)r;
        long long k = (((long long)(l / D) * D + rr / D) * D + d / D) * D + u / D;
        long long b = (((long long)(l % D) * D + rr % D) * D + d % D) * D + u % D;
        a[e] = A[k] * A[b] + A[sA + k] * A[sA + b];
    }
}

int build_double_layers(Ctx& c, double* const* sites, int Dsite)
{
    if (Dsite * Dsite != c.leg) return TN_EINVAL;
    const long long total = (long long)c.leg * c.leg * c.leg * c.leg;
    int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 8);
    for (int t = 0; t < c.nt; ++t) {
        double_layer_kernel<<<blocks, 256, 0, c.st>>>(sites[t], c.a[0][t], Dsite);
        TN_LAUNCHED();
    }
    return ctx_build_network_views(c);
}

// ============================================================================
// leg multiplication on rank-5 site tensors: out[.., j, ..] = sum_i in[.., i, ..] M[i][j]
// ============================================================================
__global__ void leg_mul_kernel(const double* __restrict__ in, double* __restrict__ out,
                               int d0, int d1, int d2, int d3, int d4, int axis,
                               const double* __restrict__ M, int nj)
{
    int din[5] = {d0, d1, d2, d3, d4};
    int dout[5] = {d0, d1, d2, d3, d4};
    dout[axis] = nj;
    long long total = 1;
    for (int k = 0; k < 5; ++k) total *= dout[k];
    long long stride_in[5];
    stride_in[4] = 1;
    for (int k = 3; k >= 0; --k) stride_in[k] = stride_in[k + 1] * din[k + 1];
    const int ni = din[axis];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long r = e, base = 0;
        int j = 0;
        for (int k = 4; k >= 0; --k) {
            int idx = (int)(r % dout[k]);
            r /= dout[k];
            if (k == axis) j = idx; else base += idx * stride_in[k];
        }
        double acc = 0.0;
        for (int i = 0; i < ni; ++i) acc = fma(in[base + i * stride_in[axis]], M[i * nj + j], acc);
        out[e] = acc;
    }
}

static int leg_mul(Ctx& c, const double* in, double* out, const int* dims, int axis, const double* M, int nj)
{
    long long total = 1;
    for (int k = 0; k < 5; ++k) total *= (k == axis ? nj : dims[k]);
    int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 4);
    leg_mul_kernel<<<blocks, 256, 0, c.st>>>(in, out, dims[0], dims[1], dims[2], dims[3], dims[4], axis, M, nj);
    TN_LAUNCHED();
    return TN_OK;
}

// Link bookkeeping shared by the small kernels.  Legs 0..3 = l, r, d, u (tensor
// axes 1..4).  Link types: (t, h) -> t, (t, v) -> nt + t.
struct Links {
    int nt, nl;
    int link_of[MAXT][4];      // link type of each leg
    int is_out[MAXT][4];       // 1 for r and d
    int out_t[MAXL], out_leg[MAXL], in_t[MAXL], in_leg[MAXL];
};

static Links make_links(const Ctx& c)
{
    Links L;
    L.nt = c.nt; L.nl = c.nl;
    for (int t = 0; t < c.nt; ++t) {
        int left = c.nt == 2 ? 1 - t : 0, up = c.nt == 2 ? 1 - t : 0;
        L.link_of[t][0] = left;           L.is_out[t][0] = 0;
        L.link_of[t][1] = t;              L.is_out[t][1] = 1;
        L.link_of[t][2] = c.nt + t;       L.is_out[t][2] = 1;
        L.link_of[t][3] = c.nt + up;      L.is_out[t][3] = 0;
    }
    for (int t = 0; t < c.nt; ++t)
        for (int g = 0; g < 4; ++g) {
            int e = L.link_of[t][g];
            if (L.is_out[t][g]) { L.out_t[e] = t; L.out_leg[e] = g; }
            else { L.in_t[e] = t; L.in_leg[e] = g; }
        }
    return L;
}

// --------------------------------------------------------------------------
// device helpers for the one-block kernels (tensors of shape [s][l][r][d][u])
// --------------------------------------------------------------------------
// Gram of T (dims 2 x n^4) on leg g with weights wt[leg][i] multiplied on the
// other legs (wt == nullptr: none): V[i][i'] = sum T[..i..] T[..i'..] prod w.
__device__ void dev_gram(const double* T, int n, int g, const double* const* wt, double* V)
{
    const int st[5] = {n * n * n * n, n * n * n, n * n, n, 1};
    int oth[3], k = 0;
    for (int leg = 0; leg < 4; ++leg) if (leg != g) oth[k++] = leg;
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int i = p / n, ip = p % n;
        double acc = 0.0;
        for (int s = 0; s < 2; ++s)
            for (int o0 = 0; o0 < n; ++o0)
                for (int o1 = 0; o1 < n; ++o1)
                    for (int o2 = 0; o2 < n; ++o2) {
                        int base = s * st[0] + o0 * st[1 + oth[0]] + o1 * st[1 + oth[1]] + o2 * st[1 + oth[2]];
                        double w = wt ? wt[oth[0]][o0] * wt[oth[1]][o1] * wt[oth[2]][o2] : 1.0;
                        acc = fma(T[base + i * st[1 + g]] * w, T[base + ip * st[1 + g]], acc);
                    }
        V[p] = acc;
    }
    __syncthreads();
}

// out = in x_leg M  (in: dims 2 x n^4; the leg g takes dimension nj), block-wide
__device__ void dev_leg_mul(const double* in, double* out, int n, int g, const double* M, int nj)
{
    int dout[5] = {2, n, n, n, n};
    dout[1 + g] = nj;
    const int total = dout[0] * dout[1] * dout[2] * dout[3] * dout[4];
    const int sin_[5] = {n * n * n * n, n * n * n, n * n, n, 1};
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int r = e, base = 0, j = 0;
        for (int k = 4; k >= 0; --k) {
            int idx = r % dout[k];
            r /= dout[k];
            if (k == 1 + g) j = idx; else base += idx * sin_[k];
        }
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc = fma(in[base + i * sin_[1 + g]], M[i * nj + j], acc);
        out[e] = acc;
    }
    __syncthreads();
}

__device__ double dev_norm(const double* x, int n, double* red)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fma(x[i], x[i], acc);
    return sqrt(block_sum(acc, red));
}

__device__ double dev_maxabs(const double* x, int n, double* red)
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
    double v = red[0];
    __syncthreads();
    return v;
}

__device__ void dev_scale(double* x, int n, double s)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] *= s;
    __syncthreads();
}

// C (row-major n x p) = A (row-major n x m) B (row-major m x p)
__device__ void dev_mm(const double* A, const double* B, double* C, int n, int m, int p)
{
    for (int e = threadIdx.x; e < n * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(A[i * m + k], B[k * p + j], acc);
        C[e] = acc;
    }
    __syncthreads();
}

// ============================================================================
// a11: canonical form (Sec. IV.A, Fig. 11), one block for the whole cell
// ============================================================================
struct CanonArgs {
    const double* A[MAXT];
    double* Aout[MAXT];
    double* lam[MAXL];
    double* maps[MAXT][4];
    Links L;
    int D;
    double tol;
    int max_iter;
    int* iters;
    double* delta;
};

__global__ void __launch_bounds__(256) canon_kernel(CanonArgs a)
{
    extern __shared__ double sm[];
    const int D = a.D, D2 = D * D, nT = 2 * D2 * D2, nt = a.L.nt, nl = a.L.nl;
    double* G = sm;                          // nt * nT
    double* Gt = G + nt * nT;                // nt * nT (ping-pong)
    double* lam = Gt + nt * nT;              // nl * D
    double* lamn = lam + nl * D;             // nl * D
    double* acc = lamn + nl * D;             // nt * 4 * D2
    double* mp = acc + nt * 4 * D2;          // nt * 4 * D2
    double* Vo = mp + nt * 4 * D2;           // D2
    double* Vi = Vo + D2;
    double* Wa = Vi + D2;
    double* Wb = Wa + D2;
    double* wa = Wb + D2;                    // D
    double* wb = wa + D;
    double* Y = wb + D;                      // D2
    double* Yi = Y + D2;
    double* Xm = Yi + D2;
    double* Xi = Xm + D2;
    double* B = Xi + D2;
    double* U = B + D2;
    double* Vs = U + D2;
    double* S = Vs + D2;                     // D
    double* ea = S + D;                      // D2 (eigh scratch)
    double* cs = ea + D2;                    // 2*(D/2+1)
    double* key = cs + 2 * (D / 2 + 1);      // D
    double* wts = key + D;                   // 4*D
    int* pq = (int*)(wts + 4 * D);           // 2*(D/2+1)
    __shared__ double red[32];
    __shared__ int flag;
    __shared__ int done;

    for (int t = 0; t < nt; ++t)
        for (int e = threadIdx.x; e < nT; e += blockDim.x) G[t * nT + e] = a.A[t][e];
    for (int e = threadIdx.x; e < nl * D; e += blockDim.x) lam[e] = 1.0 / sqrt((double)D);
    for (int e = threadIdx.x; e < nt * 4 * D2; e += blockDim.x) acc[e] = ((e % D2) / D == (e % D2) % D) ? 1.0 : 0.0;
    __syncthreads();
    int it = 0;
    double delta = 0.0;
    for (it = 1; it <= a.max_iter; ++it) {
        for (int e = 0; e < nl; ++e) {
            for (int side = 0; side < 2; ++side) {
                const int t = side == 0 ? a.L.out_t[e] : a.L.in_t[e];
                const int g = side == 0 ? a.L.out_leg[e] : a.L.in_leg[e];
                for (int q = threadIdx.x; q < 4 * D; q += blockDim.x) {
                    int leg = q / D, i = q % D;
                    wts[q] = lam[a.L.link_of[t][leg] * D + i];
                }
                __syncthreads();
                const double* w4[4] = {wts, wts + D, wts + 2 * D, wts + 3 * D};
                // weights enter squared in the Gram (lambda on each other leg of both layers)
                for (int q = threadIdx.x; q < 4 * D; q += blockDim.x) wts[q] *= wts[q];
                __syncthreads();
                dev_gram(G + t * nT, D, g, w4, side == 0 ? Vo : Vi);
            }
            dev_eigh(Vo, D, ea, wa, Wa, cs, pq, red);
            dev_eigh(Vi, D, ea, wb, Wb, cs, pq, red);
            const double ma = fmax(wa[D - 1], 0.0), mb = fmax(wb[D - 1], 0.0);
            for (int q = threadIdx.x; q < D2; q += blockDim.x) {
                int i = q / D, j = q % D;
                double ri = sqrt(fmax(wa[i], 0.0)), rj = sqrt(fmax(wa[j], 0.0));
                Y[q] = ri * Wa[i * D + j];                          // Y = D^{1/2} W^T
                double invj = (wa[j] >= 1e-14 * ma && wa[j] > 0.0) ? 1.0 / rj : 0.0;
                Yi[q] = Wa[j * D + i] * invj;                       // Y^{-1} = W D^{-1/2}
                double bj = sqrt(fmax(wb[j], 0.0));
                Xm[q] = Wb[j * D + i] * bj;                         // X = W' D'^{1/2}
                double bi = sqrt(fmax(wb[i], 0.0));
                double invi = (wb[i] >= 1e-14 * mb && wb[i] > 0.0) ? 1.0 / bi : 0.0;
                Xi[q] = invi * Wb[i * D + j];                       // X^{-1} = D'^{-1/2} W'^T
            }
            __syncthreads();
            for (int q = threadIdx.x; q < D2; q += blockDim.x) {    // B = Y diag(lambda) X
                int i = q / D, j = q % D;
                double s = 0.0;
                for (int k = 0; k < D; ++k) s = fma(Y[i * D + k] * lam[e * D + k], Xm[k * D + j], s);
                B[q] = s;
            }
            __syncthreads();
            dev_svd(B, D, D, U, S, Vs, key, &flag);
            double nrm = 0.0;
            for (int k = 0; k < D; ++k) nrm += S[k] * S[k];
            nrm = sqrt(nrm);
            for (int k = threadIdx.x; k < D; k += blockDim.x) lamn[e * D + k] = nrm > 0.0 ? S[k] / nrm : S[k];
            const int t = a.L.out_t[e], g = a.L.out_leg[e], tq = a.L.in_t[e], gq = a.L.in_leg[e];
            for (int q = threadIdx.x; q < D2; q += blockDim.x) {
                int i = q / D, j = q % D;
                double s1 = 0.0, s2 = 0.0;
                for (int k = 0; k < D; ++k) {
                    s1 = fma(Yi[i * D + k], U[j * D + k], s1);          // (Y^{-1} U)[i][j]
                    s2 = fma(Xi[k * D + i], Vs[j * D + k], s2);         // (X^{-T} V)[i][j]
                }
                mp[(t * 4 + g) * D2 + q] = s1;
                mp[(tq * 4 + gq) * D2 + q] = s2;
            }
            __syncthreads();
        }
        // apply the maps to every tensor, normalise; accumulate the maps
        for (int t = 0; t < nt; ++t) {
            double* x = G + t * nT;
            double* y = Gt + t * nT;
            dev_leg_mul(x, y, D, 0, mp + (t * 4 + 0) * D2, D);
            dev_leg_mul(y, x, D, 1, mp + (t * 4 + 1) * D2, D);
            dev_leg_mul(x, y, D, 2, mp + (t * 4 + 2) * D2, D);
            dev_leg_mul(y, x, D, 3, mp + (t * 4 + 3) * D2, D);
            double nr = dev_norm(x, nT, red);
            dev_scale(x, nT, nr > 0.0 ? 1.0 / nr : 1.0);
            for (int g = 0; g < 4; ++g) {
                double* A0 = acc + (t * 4 + g) * D2;
                dev_mm(A0, mp + (t * 4 + g) * D2, Vo, D, D, D);
                double m = dev_maxabs(Vo, D2, red);
                for (int q = threadIdx.x; q < D2; q += blockDim.x) A0[q] = m > 0.0 ? Vo[q] / m : Vo[q];
                __syncthreads();
            }
        }
        {   // every thread evaluates the (short) maximum itself
            double v = 0.0;
            for (int q = 0; q < nl * D; ++q) v = fmax(v, fabs(lamn[q] - lam[q]));
            delta = v;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nl * D; q += blockDim.x) lam[q] = lamn[q];
        if (threadIdx.x == 0) done = delta < a.tol ? 1 : 0;
        __syncthreads();
        if (done) break;
    }
    if (it > a.max_iter) it = a.max_iter;
    // weighted form sqrt(lambda) on every leg, unit norm; maps with sqrt(lambda)
    for (int t = 0; t < nt; ++t) {
        double* x = G + t * nT;
        double* y = Gt + t * nT;
        for (int g = 0; g < 4; ++g) {
            const int e = a.L.link_of[t][g];
            for (int q = threadIdx.x; q < D2; q += blockDim.x) {
                int i = q / D, j = q % D;
                Vo[q] = (i == j) ? sqrt(lam[e * D + i]) : 0.0;
            }
            __syncthreads();
            dev_leg_mul(g % 2 == 0 ? x : y, g % 2 == 0 ? y : x, D, g, Vo, D);
            dev_mm(acc + (t * 4 + g) * D2, Vo, a.maps[t][g], D, D, D);
        }
        double nr = dev_norm(x, nT, red);
        for (int e = threadIdx.x; e < nT; e += blockDim.x) a.Aout[t][e] = x[e] / nr;
    }
    for (int q = threadIdx.x; q < nl * D; q += blockDim.x) a.lam[q / D][q % D] = lam[q];
    if (threadIdx.x == 0) { *a.iters = it; *a.delta = delta; }
}

static size_t canon_smem(int D, int nt, int nl)
{
    const size_t D2 = (size_t)D * D, nT = 2 * D2 * D2;
    size_t n = 2 * nt * nT + 2 * nl * D + 2 * nt * 4 * D2 + 12 * D2 + 6 * D + 2 * (D / 2 + 1) + 4 * D;
    return n * sizeof(double) + 2 * (D / 2 + 1) * sizeof(int) + 64;
}

int canonicalize(Ctx& c, double* const* A, double* const* Aout, int* iters, bool keep_maps)
{
    (void)keep_maps;
    CanonArgs a;
    for (int t = 0; t < c.nt; ++t) {
        a.A[t] = A[t]; a.Aout[t] = Aout[t];
        for (int g = 0; g < 4; ++g) a.maps[t][g] = c.cmaps[t][g];
    }
    for (int e = 0; e < c.nl; ++e) a.lam[e] = c.lam[e];
    a.L = make_links(c);
    a.D = c.D;
    a.tol = 1e-12;
    a.max_iter = 1000;
    int* di = (int*)c.dscratch;
    a.iters = di;
    a.delta = c.dscratch + 1;
    size_t smem = canon_smem(c.D, c.nt, c.nl);
    static std::atomic<unsigned long long> attr{0};
    TN_CUDA(tn_smem_optin(canon_kernel, 200 * 1024, attr));
    if (smem > 200 * 1024) return TN_EINVAL;
    canon_kernel<<<1, 256, smem, c.st>>>(a);
    TN_LAUNCHED();
    if (iters) {
        int h = 0;
        TN_CUDA(cudaMemcpyAsync(&h, di, sizeof(int), cudaMemcpyDeviceToHost, c.st));
        TN_CUDA(cudaStreamSynchronize(c.st));
        *iters = h;
    }
    return TN_OK;
}

// ============================================================================
// a7: simple-update pre-truncation, one block per link type
// ============================================================================
// Gram of the global tensor T (2 x n^4, n = kappa*D) on leg g with the weight
// lam_{leg}[i % D] on every other leg (sqrt(lambda) on both layers).
__device__ void dev_gram_w(const double* T, int n, int D, int g, const double* const* lamw, double* V)
{
    const int st[5] = {n * n * n * n, n * n * n, n * n, n, 1};
    int oth[3], k = 0;
    for (int leg = 0; leg < 4; ++leg) if (leg != g) oth[k++] = leg;
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int i = p / n, ip = p % n;
        double acc = 0.0;
        for (int s = 0; s < 2; ++s)
            for (int o0 = 0; o0 < n; ++o0)
                for (int o1 = 0; o1 < n; ++o1)
                    for (int o2 = 0; o2 < n; ++o2) {
                        int base = s * st[0] + o0 * st[1 + oth[0]] + o1 * st[1 + oth[1]] + o2 * st[1 + oth[2]];
                        double w = lamw[oth[0]][o0 % D] * lamw[oth[1]][o1 % D] * lamw[oth[2]][o2 % D];
                        acc = fma(T[base + i * st[1 + g]] * w, T[base + ip * st[1 + g]], acc);
                    }
        V[p] = acc;
    }
    __syncthreads();
}

struct PreArgs {
    const double* Theta[MAXT];
    const double* lam[MAXL];
    double* P[MAXL];
    double* Q[MAXL];
    Links L;
    int D;
};

__global__ void __launch_bounds__(256) pretrunc_kernel(PreArgs a)
{
    extern __shared__ double sm[];
    const int e = blockIdx.x, D = a.D, n = 2 * D, n2 = n * n;
    double* Gp = sm;            // n2
    double* Gq = Gp + n2;
    double* ea = Gq + n2;       // eigh scratch n2
    double* W = ea + n2;        // n2
    double* w = W + n2;         // n
    double* Rp = w + n;         // n2
    double* Lq = Rp + n2;
    double* M = Lq + n2;
    double* U = M + n2;
    double* Vs = U + n2;
    double* S = Vs + n2;        // n
    double* key = S + n;        // n
    double* cs = key + n;       // 2*(n/2+1)
    int* pq = (int*)(cs + 2 * (n / 2 + 1));
    __shared__ double red[32];
    __shared__ int flag;
    const int t = a.L.out_t[e], g = a.L.out_leg[e], tq = a.L.in_t[e], gq = a.L.in_leg[e];
    const double* lw[4];
    for (int leg = 0; leg < 4; ++leg) lw[leg] = a.lam[a.L.link_of[t][leg]];
    dev_gram_w(a.Theta[t], n, D, g, lw, Gp);
    for (int leg = 0; leg < 4; ++leg) lw[leg] = a.lam[a.L.link_of[tq][leg]];
    dev_gram_w(a.Theta[tq], n, D, gq, lw, Gq);
    for (int side = 0; side < 2; ++side) {           // symmetric PSD square roots
        dev_eigh(side == 0 ? Gp : Gq, n, ea, w, W, cs, pq, red);
        double* R = side == 0 ? Rp : Lq;
        for (int q = threadIdx.x; q < n2; q += blockDim.x) {
            int i = q / n, j = q % n;
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += W[k * n + i] * sqrt(fmax(w[k], 0.0)) * W[k * n + j];
            R[q] = acc;
        }
        __syncthreads();
    }
    dev_mm(Rp, Lq, M, n, n, n);
    dev_svd(M, n, n, U, S, Vs, key, &flag);
    const double s0 = S[0];
    for (int q = threadIdx.x; q < n * D; q += blockDim.x) {      // P = Lq V_D S^{-1/2}
        int i = q / D, j = q % D;
        double inv = (s0 > 0.0 && S[j] >= 1e-12 * s0) ? 1.0 / sqrt(S[j]) : 0.0;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = fma(Lq[i * n + k], Vs[j * n + k], acc);
        a.P[e][q] = acc * inv;
    }
    for (int q = threadIdx.x; q < D * n; q += blockDim.x) {      // Q = S^{-1/2} U_D^T Rp
        int i = q / n, j = q % n;
        double inv = (s0 > 0.0 && S[i] >= 1e-12 * s0) ? 1.0 / sqrt(S[i]) : 0.0;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = fma(U[i * n + k], Rp[k * n + j], acc);
        a.Q[e][q] = acc * inv;
    }
}

// ============================================================================
// a8: PSD projection of the bond environment (one block per link type)
//     N4[a][b][a'][b'] -> matrix [(a,b)][(a',b')], divided by <g|g> = sum N4[c][c][e][e],
//     symmetrised, negative eigenvalues clipped.  empty[e] = 1 if <g|g> == 0.
// ============================================================================
__global__ void __launch_bounds__(512) psd_kernel(double* N4all, int kD, int* empty)
{
    extern __shared__ double sm[];
    const int n = kD * kD, n2 = n * n;
    double* N4 = N4all + (size_t)blockIdx.x * n2;
    double* A = sm;           // n2
    double* V = A + n2;       // n2
    double* w = V + n2;       // n
    double* cs = w + n;       // 2*(n/2+1)
    int* pq = (int*)(cs + 2 * (n / 2 + 1));
    __shared__ double red[32];
    double tr = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        int c = q / kD, e = q % kD;
        tr += N4[(size_t)(c * kD + c) * n + (e * kD + e)];
    }
    tr = block_sum(tr, red);
    if (!(fabs(tr) > 0.0)) {
        if (threadIdx.x == 0) empty[blockIdx.x] = 1;
        return;
    }
    if (threadIdx.x == 0) empty[blockIdx.x] = 0;
    dev_eigh(N4, n, A, w, V, cs, pq, red);
    for (int q = threadIdx.x; q < n2; q += blockDim.x) {
        int i = q / n, j = q % n;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += V[k * n + i] * fmax(w[k] / tr, 0.0) * V[k * n + j];
        N4[q] = acc;
    }
}

// ============================================================================
// a9: ALS of Eq. (var1) with a pseudo-inverse, then balancing (one block per link)
// ============================================================================
// x = R^+ rhs through the eigenvalues of R; those below cut * max are dropped
// (the ALS of a9 passes cut = 1e-12)
__device__ void dev_pinv_solve(const double* R, int n, const double* rhs, double* x, double* A, double* W,
                               double* w, double* cs, int* pq, double* red, double* tmp, double cut)
{
    dev_eigh(R, n, A, w, W, cs, pq, red);
    const double wm = w[n - 1];
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc = fma(W[k * n + i], rhs[i], acc);
        tmp[k] = (wm > 0.0 && w[k] >= cut * wm) ? acc / w[k] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = fma(W[k * n + i], tmp[k], acc);
        x[i] = acc;
    }
    __syncthreads();
}

struct AlsArgs {
    const double* N4;      // per link (kD)^4, stride (kD)^4
    const int* empty;
    const double* P0[MAXL];
    const double* Q0[MAXL];
    double* P[MAXL];
    double* Q[MAXL];
    int* iters;
    double* cost;
    int D;
    double tol;
    int max_iter;
    double cut;            // relative pseudo-inverse cutoff of the normal equations
};

__global__ void __launch_bounds__(256) als_kernel(AlsArgs a)
{
    extern __shared__ double sm[];
    const int e = blockIdx.x, D = a.D, k = 2 * D, k2 = k * k, nR = k * D;
    double* N4 = sm;                 // k^4
    double* n2 = N4 + k2 * k2;       // k2
    double* P = n2 + k2;             // k*D
    double* Q = P + nR;              // D*k
    double* Mo = Q + nR;             // k2
    double* Mn = Mo + k2;            // k2
    double* R = Mn + k2;             // nR^2
    double* A = R + nR * nR;         // nR^2
    double* W = A + nR * nR;         // nR^2
    double* w = W + nR * nR;         // nR
    double* rhs = w + nR;            // nR
    double* x = rhs + nR;            // nR
    double* tmp = x + nR;            // nR
    double* cs = tmp + nR;           // 2*(nR/2+1)
    int* pq = (int*)(cs + 2 * (nR / 2 + 1));
    __shared__ double red[32];
    __shared__ int flag;
    __shared__ int stop;
    const bool empty = a.empty[e] != 0;
    for (int q = threadIdx.x; q < nR; q += blockDim.x) { P[q] = a.P0[e][q]; Q[q] = a.Q0[e][q]; }
    if (empty) {
        __syncthreads();
        for (int q = threadIdx.x; q < nR; q += blockDim.x) { a.P[e][q] = P[q]; a.Q[e][q] = Q[q]; }
        if (threadIdx.x == 0) { a.iters[e] = 0; a.cost[e] = NAN; }
        return;
    }
    for (int q = threadIdx.x; q < k2 * k2; q += blockDim.x) N4[q] = a.N4[(size_t)e * k2 * k2 + q];
    __syncthreads();
    for (int q = threadIdx.x; q < k2; q += blockDim.x) {        // n2[a][b] = sum_c N4[a][b][c][c]
        double acc = 0.0;
        for (int c = 0; c < k; ++c) acc += N4[q * k2 + c * k + c];
        n2[q] = acc;
    }
    __syncthreads();
    dev_mm(P, Q, Mo, k, D, k);
    int it = 0;
    for (it = 1; it <= a.max_iter; ++it) {
        // P-step: R[(a,i)][(a',i')] = sum_{b,b'} Q[i][b] Q[i'][b'] N4[a][b][a'][b']
        for (int q = threadIdx.x; q < nR * nR; q += blockDim.x) {
            int r1 = q / nR, r2 = q % nR;
            int aa = r1 / D, i = r1 % D, ap = r2 / D, ip = r2 % D;
            double acc = 0.0;
            for (int b = 0; b < k; ++b)
                for (int bp = 0; bp < k; ++bp)
                    acc = fma(Q[i * k + b] * Q[ip * k + bp], N4[((aa * k + b) * k + ap) * k + bp], acc);
            R[q] = acc;
        }
        for (int q = threadIdx.x; q < nR; q += blockDim.x) {
            int aa = q / D, i = q % D;
            double acc = 0.0;
            for (int b = 0; b < k; ++b) acc = fma(Q[i * k + b], n2[aa * k + b], acc);
            rhs[q] = acc;
        }
        __syncthreads();
        dev_pinv_solve(R, nR, rhs, P, A, W, w, cs, pq, red, tmp, a.cut);     // P[(a,i)]
        // Q-step: R[(i,b)][(i',b')] = sum_{a,a'} P[a][i] P[a'][i'] N4[a][b][a'][b']
        for (int q = threadIdx.x; q < nR * nR; q += blockDim.x) {
            int r1 = q / nR, r2 = q % nR;
            int i = r1 / k, b = r1 % k, ip = r2 / k, bp = r2 % k;
            double acc = 0.0;
            for (int aa = 0; aa < k; ++aa)
                for (int ap = 0; ap < k; ++ap)
                    acc = fma(P[aa * D + i] * P[ap * D + ip], N4[((aa * k + b) * k + ap) * k + bp], acc);
            R[q] = acc;
        }
        for (int q = threadIdx.x; q < nR; q += blockDim.x) {
            int i = q / k, b = q % k;
            double acc = 0.0;
            for (int aa = 0; aa < k; ++aa) acc = fma(P[aa * D + i], n2[aa * k + b], acc);
            rhs[q] = acc;
        }
        __syncthreads();
        dev_pinv_solve(R, nR, rhs, Q, A, W, w, cs, pq, red, tmp, a.cut);     // Q[(i,b)]
        dev_mm(P, Q, Mn, k, D, k);
        double dm = 0.0, mn = 0.0;
        for (int q = 0; q < k2; ++q) { double d = Mn[q] - Mo[q]; dm += d * d; mn += Mn[q] * Mn[q]; }
        __syncthreads();
        for (int q = threadIdx.x; q < k2; q += blockDim.x) Mo[q] = Mn[q];
        if (threadIdx.x == 0) stop = (sqrt(dm) <= a.tol * sqrt(mn)) ? 1 : 0;
        __syncthreads();
        if (stop) break;
    }
    if (it > a.max_iter) it = a.max_iter;
    // cost f = T - 2 <M, n2> + <M (x) M, N4>, T = sum N4[c][c][e][e]
    double part = 0.0;
    for (int q = threadIdx.x; q < k2 * k2; q += blockDim.x) {
        int bp = q % k, ap = (q / k) % k, b = (q / k2) % k, aa = q / (k2 * k);
        part += Mo[aa * k + b] * Mo[ap * k + bp] * N4[q];
        if (aa == b && ap == bp) part += N4[q];
    }
    for (int q = threadIdx.x; q < k2; q += blockDim.x) part -= 2.0 * Mo[q] * n2[q];
    double f = block_sum(part, red);
    // balance: M = U S V^T, P = U_D sqrt(S), Q = sqrt(S) V_D^T
    double* U = R;              // reuse: k2
    double* Vb = A;             // k2
    double* S = w;              // k
    double* key = rhs;          // k
    dev_svd(Mo, k, k, U, S, Vb, key, &flag);
    for (int q = threadIdx.x; q < k * D; q += blockDim.x) {
        int i = q / D, j = q % D;
        a.P[e][q] = U[j * k + i] * sqrt(S[j]);
    }
    for (int q = threadIdx.x; q < D * k; q += blockDim.x) {
        int i = q / k, j = q % k;
        a.Q[e][q] = sqrt(S[i]) * Vb[i * k + j];
    }
    if (threadIdx.x == 0) { a.iters[e] = it; a.cost[e] = f; }
}

// ============================================================================
// a12: gauge fixing by local fidelity (Sec. IV.B, Eq. 25), one block per cell
// ============================================================================
struct GaugeArgs {
    const double* A0[MAXT];
    const double* B[MAXT];
    const double* P[MAXL];          // full-update pairs and canonical maps: the starting W
    const double* Q[MAXL];
    const double* maps[MAXT][4];
    double* W[MAXL];
    double* F;
    int* iters;
    Links L;
    int D;
    double tol;
    int max_iter;
};

__global__ void __launch_bounds__(256) gauge_kernel(GaugeArgs a)
{
    extern __shared__ double sm[];
    const int D = a.D, D2 = D * D, nT = 2 * D2 * D2, nt = a.L.nt, nl = a.L.nl;
    double* A0 = sm;                  // nt*nT
    double* B = A0 + nt * nT;         // nt*nT
    double* X = B + nt * nT;          // nT
    double* Y = X + nT;               // nT
    double* W = Y + nT;               // nl*D2
    double* M = W + nl * D2;          // D2
    double* U = M + D2;
    double* Vs = U + D2;
    double* S = Vs + D2;              // D
    double* key = S + D;              // D
    __shared__ double red[32];
    __shared__ int flag;
    __shared__ int stop;
    for (int t = 0; t < nt; ++t)
        for (int q = threadIdx.x; q < nT; q += blockDim.x) { A0[t * nT + q] = a.A0[t][q]; B[t * nT + q] = a.B[t][q]; }
    // start: W_e = polar(sum over the link's legs of the kappa = 0 rows of P Q_c (out) or Q^T Q_c (in))
    for (int e = 0; e < nl; ++e) {
        for (int p = threadIdx.x; p < D2; p += blockDim.x) {
            int i = p / D, j = p % D;
            double acc = 0.0;
            for (int t = 0; t < nt; ++t)
                for (int g = 0; g < 4; ++g) {
                    if (a.L.link_of[t][g] != e) continue;
                    const double* mp = a.maps[t][g];
                    for (int l = 0; l < D; ++l) {
                        double b = a.L.is_out[t][g] ? a.P[e][i * D + l] : a.Q[e][l * 2 * D + i];
                        acc = fma(b, mp[l * D + j], acc);
                    }
                }
            M[p] = acc;
        }
        __syncthreads();
        dev_svd(M, D, D, U, S, Vs, key, &flag);
        for (int p = threadIdx.x; p < D2; p += blockDim.x) {
            int i = p / D, j = p % D;
            double acc = 0.0;
            for (int q = 0; q < D; ++q) acc = fma(U[q * D + i], Vs[q * D + j], acc);
            W[e * D2 + p] = acc;
        }
        __syncthreads();
    }
    int it = 0;
    for (it = 1; it <= a.max_iter; ++it) {
        double change = 0.0;
        for (int e = 0; e < nl; ++e) {
            for (int q = threadIdx.x; q < D2; q += blockDim.x) M[q] = 0.0;
            __syncthreads();
            for (int t = 0; t < nt; ++t)
                for (int g = 0; g < 4; ++g) {
                    if (a.L.link_of[t][g] != e) continue;
                    // X = A0_t with every other leg transformed
                    const double* src = A0 + t * nT;
                    double* bufs[2] = {X, Y};
                    int cur = -1;
                    for (int o = 0; o < 4; ++o) {
                        if (o == g) continue;
                        double* dst = bufs[(cur + 1) & 1];
                        dev_leg_mul(cur < 0 ? src : bufs[cur & 1], dst, D, o, W + a.L.link_of[t][o] * D2, D);
                        cur = (cur + 1) & 1;
                    }
                    const double* Xt = bufs[cur & 1];
                    // M[i][j] += sum_rest Xt[..i..] B_t[..j..] on leg g
                    const int st[5] = {D2 * D2, D2 * D, D2, D, 1};
                    int oth[3], kk = 0;
                    for (int leg = 0; leg < 4; ++leg) if (leg != g) oth[kk++] = leg;
                    for (int p = threadIdx.x; p < D2; p += blockDim.x) {
                        int i = p / D, j = p % D;
                        double acc = 0.0;
                        for (int s = 0; s < 2; ++s)
                            for (int o0 = 0; o0 < D; ++o0)
                                for (int o1 = 0; o1 < D; ++o1)
                                    for (int o2 = 0; o2 < D; ++o2) {
                                        int base = s * st[0] + o0 * st[1 + oth[0]] + o1 * st[1 + oth[1]] + o2 * st[1 + oth[2]];
                                        acc = fma(Xt[base + i * st[1 + g]], B[t * nT + base + j * st[1 + g]], acc);
                                    }
                        M[p] += acc;
                    }
                    __syncthreads();
                }
            dev_svd(M, D, D, U, S, Vs, key, &flag);
            double ch = 0.0;
            for (int p = 0; p < D2; ++p) {           // W = U V^T (every thread, D2 small)
                int i = p / D, j = p % D;
                double acc = 0.0;
                for (int q = 0; q < D; ++q) acc = fma(U[q * D + i], Vs[q * D + j], acc);
                ch = fmax(ch, fabs(acc - W[e * D2 + p]));
            }
            __syncthreads();
            for (int p = threadIdx.x; p < D2; p += blockDim.x) {
                int i = p / D, j = p % D;
                double acc = 0.0;
                for (int q = 0; q < D; ++q) acc = fma(U[q * D + i], Vs[q * D + j], acc);
                W[e * D2 + p] = acc;
            }
            __syncthreads();
            change = fmax(change, ch);
        }
        if (threadIdx.x == 0) stop = change < a.tol ? 1 : 0;
        __syncthreads();
        if (stop) break;
    }
    if (it > a.max_iter) it = a.max_iter;
    double Fsum = 0.0;
    for (int t = 0; t < nt; ++t) {
        const double* src = A0 + t * nT;
        dev_leg_mul(src, X, D, 0, W + a.L.link_of[t][0] * D2, D);
        dev_leg_mul(X, Y, D, 1, W + a.L.link_of[t][1] * D2, D);
        dev_leg_mul(Y, X, D, 2, W + a.L.link_of[t][2] * D2, D);
        dev_leg_mul(X, Y, D, 3, W + a.L.link_of[t][3] * D2, D);
        double part = 0.0;
        for (int q = threadIdx.x; q < nT; q += blockDim.x) part = fma(Y[q], B[t * nT + q], part);
        Fsum += block_sum(part, red);
    }
    for (int q = threadIdx.x; q < nl * D2; q += blockDim.x) a.W[q / D2][q % D2] = W[q];
    if (threadIdx.x == 0) { *a.F = Fsum / nt; *a.iters = it; }
}

// ============================================================================
// a13: renormalised-gate leg matrices K = base . maps . W^T (kappa*D x D)
// ============================================================================
struct GateArgs {
    const double* base[MAXT][4];   // P (out legs) or Q (in legs, used transposed)
    int transposed[MAXT][4];
    const double* maps[MAXT][4];
    const double* W[MAXT][4];
    double* K[MAXT][4];
    int D;
};

__global__ void gate_kernel(GateArgs a)
{
    const int t = blockIdx.x / 4, g = blockIdx.x % 4, D = a.D, k = 2 * D;
    __shared__ double T1[16 * 8];
    for (int q = threadIdx.x; q < k * D; q += blockDim.x) {       // T1 = base . maps
        int i = q / D, j = q % D;
        double acc = 0.0;
        for (int l = 0; l < D; ++l) {
            double b = a.transposed[t][g] ? a.base[t][g][l * k + i] : a.base[t][g][i * D + l];
            acc = fma(b, a.maps[t][g][l * D + j], acc);
        }
        T1[q] = acc;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < k * D; q += blockDim.x) {       // K = T1 . W^T
        int i = q / D, j = q % D;
        double acc = 0.0;
        for (int l = 0; l < D; ++l) acc = fma(T1[i * D + l], a.W[t][g][j * D + l], acc);
        a.K[t][g][q] = acc;
    }
}

// ============================================================================
// a14: expectation values from the reduced density matrices
// ============================================================================
__global__ void expect_kernel(const double* rho1, int nt, const double* rho2, int nl, double J, double h, double* out)
{
    if (threadIdx.x != 0) return;
    // out: [e_site, e_link, mx[2], mz[2], zz[4]]
    double sx = 0.0, szz = 0.0;
    for (int t = 0; t < nt; ++t) {
        const double* r = rho1 + 4 * t;           // r[s][s']
        double tr = r[0] + r[3];
        double mx = (r[1] + r[2]) / tr;            // Tr(rho X)
        double mz = (r[0] - r[3]) / tr;            // Tr(rho Z)
        out[2 + t] = mx; out[4 + t] = mz;
        sx += mx;
    }
    for (int e = 0; e < nl; ++e) {
        const double* r = rho2 + 16 * e;          // r[s][t][s'][t'] -> [(s t)][(s' t')]
        double tr = 0.0, zz = 0.0;
        for (int st = 0; st < 4; ++st) {
            double v = r[st * 4 + st];
            tr += v;
            int s = st >> 1, tt = st & 1;
            zz += ((s == tt) ? 1.0 : -1.0) * v;
        }
        out[6 + e] = zz / tr;
        szz += zz / tr;
    }
    double es = -J * szz / nt - h * sx / nt;
    out[0] = es; out[1] = 0.5 * es;
}

// ============================================================================
// finiteness of the state: flag = 1 if any entry is NaN or Inf
// ============================================================================
__global__ void nonfinite_kernel(const double* __restrict__ x, long long n, int* __restrict__ flag)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) *flag = 1;       // every writer stores the same value
}

int state_finite(Ctx& c, double* const* T, bool* ok)
{
    int* flag = (int*)(c.dscratch + 48);
    TN_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c.st));
    const long long n = 2LL * c.D * c.D * c.D * c.D;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152);
    for (int t = 0; t < c.nt; ++t) {
        nonfinite_kernel<<<blocks, 256, 0, c.st>>>(T[t], n, flag);
        TN_LAUNCHED();
    }
    int h = 0;
    TN_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    TN_CUDA(cudaStreamSynchronize(c.st));
    *ok = (h == 0);
    return TN_OK;
}

// ============================================================================
// host orchestration
// ============================================================================
static int apply_legs(Ctx& c, const double* T, double* out, int t, double* const* P, double* const* Q, int D_in)
{
    // out = T with every leg mapped D_in -> D (P on out legs, Q^T on in legs)
    Links L = make_links(c);
    size_t mk = c.ar.mark();
    double* b0 = c.ar.take((size_t)2 * D_in * D_in * D_in * D_in);
    double* b1 = c.ar.take((size_t)2 * D_in * D_in * D_in * D_in);
    double* Qt = c.ar.take((size_t)D_in * c.D);
    if (!b0 || !b1 || !Qt) return TN_ENOMEM;
    int dims[5] = {2, D_in, D_in, D_in, D_in};
    const double* src = T;
    double* bufs[2] = {b0, b1};
    for (int g = 0; g < 4; ++g) {
        const int e = L.link_of[t][g];
        const double* M;
        if (L.is_out[t][g]) M = P[e];
        else {
            const int pd[2] = {c.D, D_in}, pp[2] = {1, 0};
            TN_TRY(permute(c.st, Q[e], Qt, 2, pd, pp));
            M = Qt;
        }
        double* dst = (g == 3) ? out : bufs[g & 1];
        TN_TRY(leg_mul(c, src, dst, dims, 1 + g, M, c.D));
        dims[1 + g] = c.D;
        src = dst;
    }
    c.ar.release(mk);
    return TN_OK;
}

// Canonical form, Theta = g A_c and the simple-update projectors (a11, a1, a7).
static int prepare_theta(Ctx& c, int* canon_iters)
{
    if (!c.have_state) return TN_ESTATE;
    if (!c.have_pepo) return TN_ESTATE;
    bool ok = true;
    TN_TRY(state_finite(c, c.A, &ok));
    if (!ok) return TN_ENUMERIC;
    int it = 0;
    TN_TRY(canonicalize(c, c.A, c.Ac, &it, true));                      // a11
    for (int t = 0; t < c.nt; ++t) TN_TRY(apply_pepo(c, c.Ac[t], c.Theta[t]));   // a1
    PreArgs pa;                                                          // a7
    for (int t = 0; t < c.nt; ++t) pa.Theta[t] = c.Theta[t];
    for (int e = 0; e < c.nl; ++e) { pa.lam[e] = c.lam[e]; pa.P[e] = c.preP[e]; pa.Q[e] = c.preQ[e]; }
    pa.L = make_links(c);
    pa.D = c.D;
    const int n = 2 * c.D, n2 = n * n;
    size_t smem = sizeof(double) * (10 * (size_t)n2 + 3 * n + 2 * (n / 2 + 1)) + sizeof(int) * 2 * (n / 2 + 1) + 64;
    pretrunc_kernel<<<c.nl, 256, smem, c.st>>>(pa);
    TN_LAUNCHED();
    *canon_iters = it;
    return TN_OK;
}

int step_prepare(Ctx& c, tn_step_report* rep)
{
    int it = 0;
    TN_TRY(prepare_theta(c, &it));
    for (int t = 0; t < c.nt; ++t) TN_TRY(apply_legs(c, c.Theta[t], c.A1[t], t, c.preP, c.preQ, c.kD));   // A'
    if (c.leg != c.D * c.D) return TN_ESTATE;
    TN_TRY(build_double_layers(c, c.A1, c.D));                          // a2
    c.have_network = true;
    c.prepared = true;
    if (rep) rep->canon_iters = it;
    return TN_OK;
}

// Bond environment of link type e (a8): raw N[a][b][a'][b'] into out.
static int bond_env(Ctx& c, int e, double* out)
{
    const int chi = c.chi, L = c.leg, D = c.D, k = c.kD;
    Links lk = make_links(c);
    const int t = lk.out_t[e], tq = lk.in_t[e];
    const bool vertical = e >= c.nt;
    size_t mk = c.ar.mark();
    // open-leg tensors: Tp keeps its out leg at kappa*D, Tq its in leg
    double* Tp = c.ar.take((size_t)2 * k * D * D * D);
    double* Tq = c.ar.take((size_t)2 * k * D * D * D);
    double* Rp = c.ar.take((size_t)2 * k * D * D * D);
    double* Rq = c.ar.take((size_t)2 * k * D * D * D);
    double* b0 = c.ar.take((size_t)2 * k * k * k * k);
    double* b1 = c.ar.take((size_t)2 * k * k * k * k);
    double* Qt = c.ar.take((size_t)k * D);
    if (!Tp || !Tq || !Rp || !Rq || !b0 || !b1 || !Qt) return TN_ENOMEM;
    for (int side = 0; side < 2; ++side) {
        const int tt = side == 0 ? t : tq;
        const int open = side == 0 ? lk.out_leg[e] : lk.in_leg[e];
        int dims[5] = {2, k, k, k, k};
        const double* src = c.Theta[tt];
        double* bufs[2] = {b0, b1};
        int used = 0;
        for (int g = 0; g < 4; ++g) {
            if (g == open) continue;
            const int ee = lk.link_of[tt][g];
            const double* M;
            if (lk.is_out[tt][g]) M = c.preP[ee];
            else {
                const int pd[2] = {D, k}, pp[2] = {1, 0};
                TN_TRY(permute(c.st, c.preQ[ee], Qt, 2, pd, pp));
                M = Qt;
            }
            double* dst = (used == 2) ? (side == 0 ? Tp : Tq) : bufs[used & 1];
            TN_TRY(leg_mul(c, src, dst, dims, 1 + g, M, D));
            dims[1 + g] = D;
            src = dst;
            ++used;
        }
    }
    int xp, yp;
    Frame f = c.frame0();
    const int tpos[2][2] = {{0, 0}, {1, 0}};
    xp = tpos[t][0]; yp = tpos[t][1];
    if (vertical) {
        // rotate the two tensors and the frame once: the vertical link becomes horizontal
        const int dp[5] = {2, D, D, k, D}, dq[5] = {2, D, D, D, k};   // Tp: d open (axis 3); Tq: u open (axis 4)
        const int rot5[5] = {0, 4, 3, 1, 2};
        TN_TRY(permute(c.st, Tp, Rp, 5, dp, rot5));
        TN_TRY(permute(c.st, Tq, Rq, 5, dq, rot5));
        std::swap(Tp, Rp);
        std::swap(Tq, Rq);
        Frame fr = f.rotated();
        int xr = ((yp % f.Ly) + f.Ly) % f.Ly, yr = ((-xp) % f.Lx + f.Lx) % f.Lx;
        f = fr; xp = xr; yp = yr;
    }
    Env& ep = f.e(xp, yp);
    Env& eq = f.e(xp + 1, yp);
    // after rotation Tp: [s][l D][r k][d D][u D], Tq: [s][l k][r D][d D][u D]
    double* X1 = c.ar.take((size_t)chi * chi * L);
    double* X2 = c.ar.take((size_t)chi * chi * L * L);
    double* X3 = c.ar.take((size_t)chi * chi * D * D * 2 * k * D);
    double* X4 = c.ar.take((size_t)chi * chi * k * k * D * D);
    double* LL = c.ar.take((size_t)chi * chi * L);
    double* EL = c.ar.take((size_t)chi * chi * k * k);
    double* ER = c.ar.take((size_t)chi * chi * k * k);
    double* Nr = c.ar.take((size_t)k * k * k * k);
    if (!X1 || !X2 || !X3 || !X4 || !LL || !EL || !ER || !Nr) return TN_ENOMEM;
    // E_L: C1 T1 T4 (ket) (bra) C4 T3 of p
    TN_TRY(contract(c.st, c.ar, "ia,aom->iom", dt(ep.C[0], {chi, chi}), dt(ep.T[0], {chi, chi, L}), dt(X1, {chi, chi, L})));
    TN_TRY(contract(c.st, c.ar, "iom,jin->omjn", dt(X1, {chi, chi, L}), dt(ep.T[3], {chi, chi, L}), dt(X2, {chi, L, chi, L})));
    TN_TRY(contract(c.st, c.ar, "oUujLl,sLRDU->oujlsRD", dt(X2, {chi, D, D, chi, D, D}), dt(Tp, {2, D, k, D, D}),
                    dt(X3, {chi, D, chi, D, 2, k, D})));
    TN_TRY(contract(c.st, c.ar, "oujlsRD,slrdu->ojRDrd", dt(X3, {chi, D, chi, D, 2, k, D}), dt(Tp, {2, D, k, D, D}),
                    dt(X4, {chi, chi, k, D, k, D})));
    TN_TRY(contract(c.st, c.ar, "kj,nkm->jnm", dt(ep.C[3], {chi, chi}), dt(ep.T[2], {chi, chi, L}), dt(LL, {chi, chi, L})));
    TN_TRY(contract(c.st, c.ar, "ojRDrd,jnDd->onRr", dt(X4, {chi, chi, k, D, k, D}), dt(LL, {chi, chi, D, D}),
                    dt(EL, {chi, chi, k, k})));
    // E_R: T1 C2 T2 (ket) (bra) C3 T3 of q
    TN_TRY(contract(c.st, c.ar, "oam,ac->ocm", dt(eq.T[0], {chi, chi, L}), dt(eq.C[1], {chi, chi}), dt(X1, {chi, chi, L})));
    TN_TRY(contract(c.st, c.ar, "ocm,ctn->omtn", dt(X1, {chi, chi, L}), dt(eq.T[1], {chi, chi, L}), dt(X2, {chi, L, chi, L})));
    TN_TRY(contract(c.st, c.ar, "oUutRr,sLRDU->outrsLD", dt(X2, {chi, D, D, chi, D, D}), dt(Tq, {2, k, D, D, D}),
                    dt(X3, {chi, D, chi, D, 2, k, D})));
    TN_TRY(contract(c.st, c.ar, "outrsLD,slrdu->otLDld", dt(X3, {chi, D, chi, D, 2, k, D}), dt(Tq, {2, k, D, D, D}),
                    dt(X4, {chi, chi, k, D, k, D})));
    TN_TRY(contract(c.st, c.ar, "te,enm->tnm", dt(eq.C[2], {chi, chi}), dt(eq.T[2], {chi, chi, L}), dt(LL, {chi, chi, L})));
    TN_TRY(contract(c.st, c.ar, "otLDld,tnDd->onLl", dt(X4, {chi, chi, k, D, k, D}), dt(LL, {chi, chi, D, D}),
                    dt(ER, {chi, chi, k, k})));
    TN_TRY(contract(c.st, c.ar, "onAa,onBb->AaBb", dt(EL, {chi, chi, k, k}), dt(ER, {chi, chi, k, k}), dt(Nr, {k, k, k, k})));
    TN_TRY(permute_spec(c.st, "AaBb->ABab", dt(Nr, {k, k, k, k}), dt(out, {k, k, k, k})));
    c.ar.release(mk);
    return TN_OK;
}

// Simple-update step (the environment-free method the full update is compared
// with, Sec. VI.B last paragraph and Sec. VI.D): A <- Theta truncated on every
// leg by the lambda-weighted projectors of a7, max-abs normalised.
int su_step(Ctx& c, tn_step_report* rep)
{
    int it = 0;
    TN_TRY(prepare_theta(c, &it));
    for (int t = 0; t < c.nt; ++t) {
        TN_TRY(apply_legs(c, c.Theta[t], c.A[t], t, c.preP, c.preQ, c.kD));
        TN_TRY(normalize_maxabs(c.st, c.A[t], 2LL * c.D * c.D * c.D * c.D, 1, 0));
    }
    c.prepared = false;
    c.updated = false;
    if (rep) rep->canon_iters = it;
    bool ok = true;
    TN_TRY(state_finite(c, c.A, &ok));
    return ok ? TN_OK : TN_ENUMERIC;
}

// Bond environments of every link type (a8) into c.N4, normalised by <g|g>,
// symmetrised and projected on their positive part; empty[e] flags <g|g> = 0.
int bond_envs_psd(Ctx& c)
{
    if (!c.prepared) return TN_ESTATE;
    const int k = c.kD;
    for (int e = 0; e < c.nl; ++e) TN_TRY(bond_env(c, e, c.N4[e]));                    // a8
    int* empty = (int*)(c.dscratch + 8);
    {
        const int n = k * k;
        size_t smem = sizeof(double) * (2 * (size_t)n * n + n + 2 * (n / 2 + 1)) + sizeof(int) * 2 * (n / 2 + 1) + 64;
        static std::atomic<unsigned long long> attr{0};
        TN_CUDA(tn_smem_optin(psd_kernel, 200 * 1024, attr));
        if (smem > 200 * 1024) return TN_EINVAL;
        // N4 buffers are consecutive (allocated together)
        psd_kernel<<<c.nl, 512, smem, c.st>>>(c.N4[0], k, empty);
        TN_LAUNCHED();
    }
    return TN_OK;
}

int step_update(Ctx& c, tn_step_report* rep)
{
    if (!c.prepared) return TN_ESTATE;
    const int k = c.kD, n4 = k * k * k * k;
    TN_TRY(bond_envs_psd(c));                                                            // a8
    int* empty = (int*)(c.dscratch + 8);
    AlsArgs aa;                                                                          // a9
    aa.N4 = c.N4[0];
    aa.empty = empty;
    for (int e = 0; e < c.nl; ++e) { aa.P0[e] = c.preP[e]; aa.Q0[e] = c.preQ[e]; aa.P[e] = c.fuP[e]; aa.Q[e] = c.fuQ[e]; }
    int* iters = (int*)(c.dscratch + 16);
    double* cost = c.dscratch + 24;
    aa.iters = iters;
    aa.cost = cost;
    aa.D = c.D;
    aa.tol = c.als_tol;
    aa.max_iter = c.als_max;
    aa.cut = 1e-12;
    {
        const int nR = k * c.D;
        size_t smem = sizeof(double) * ((size_t)n4 + 3 * (size_t)k * k + 2 * nR + 3 * (size_t)nR * nR + 4 * nR + 2 * (nR / 2 + 1))
                      + sizeof(int) * 2 * (nR / 2 + 1) + 64;
        static std::atomic<unsigned long long> attr{0};
        TN_CUDA(tn_smem_optin(als_kernel, 200 * 1024, attr));
        if (smem > 200 * 1024) return TN_EINVAL;
        als_kernel<<<c.nl, 256, smem, c.st>>>(aa);
        TN_LAUNCHED();
    }
    for (int t = 0; t < c.nt; ++t) {                                                     // a10
        TN_TRY(apply_legs(c, c.Theta[t], c.A[t], t, c.fuP, c.fuQ, c.kD));
        TN_TRY(normalize_maxabs(c.st, c.A[t], 2LL * c.D * c.D * c.D * c.D, 1, 0));
    }
    if (rep) {
        int hi[MAXL]; double hc[MAXL];
        TN_CUDA(cudaMemcpyAsync(hi, iters, sizeof(int) * c.nl, cudaMemcpyDeviceToHost, c.st));
        TN_CUDA(cudaMemcpyAsync(hc, cost, sizeof(double) * c.nl, cudaMemcpyDeviceToHost, c.st));
        TN_CUDA(cudaStreamSynchronize(c.st));
        for (int e = 0; e < c.nl; ++e) { rep->als_iters[e] = hi[e]; rep->als_cost[e] = hc[e]; }
    }
    c.updated = true;
    c.prepared = false;
    bool ok = true;
    TN_TRY(state_finite(c, c.A, &ok));
    return ok ? TN_OK : TN_ENUMERIC;
}

// Steps (i)-(iii) of the window: A_0, canonical form of A~, gauge fix, leg
// matrices K; the state is reset to A_0.
int recycle_build(Ctx& c, double* F)
{
    if (!c.updated) return TN_ESTATE;
    const int D = c.D;
    // A_0 = A_c (the canonical state the step started from); A~ is in c.A
    for (int t = 0; t < c.nt; ++t)
        TN_CUDA(cudaMemcpyAsync(c.A0[t], c.Ac[t], sizeof(double) * 2 * D * D * D * D, cudaMemcpyDeviceToDevice, c.st));
    TN_TRY(canonicalize(c, c.A, c.A1, nullptr, true));                                    // a11 on A~
    GaugeArgs ga;                                                                         // a12
    for (int t = 0; t < c.nt; ++t) {
        ga.A0[t] = c.A0[t]; ga.B[t] = c.A1[t];
        for (int g = 0; g < 4; ++g) ga.maps[t][g] = c.cmaps[t][g];
    }
    for (int e = 0; e < c.nl; ++e) { ga.W[e] = c.W[e]; ga.P[e] = c.fuP[e]; ga.Q[e] = c.fuQ[e]; }
    ga.F = c.dscratch + 32;
    ga.iters = (int*)(c.dscratch + 33);
    ga.L = make_links(c);
    ga.D = D;
    ga.tol = 1e-12;
    ga.max_iter = 500;
    {
        const size_t D2 = (size_t)D * D, nT = 2 * D2 * D2;
        size_t smem = sizeof(double) * (2 * c.nt * nT + 2 * nT + c.nl * D2 + 4 * D2 + 2 * D) + 64;
        static std::atomic<unsigned long long> attr{0};
        TN_CUDA(tn_smem_optin(gauge_kernel, 200 * 1024, attr));
        if (smem > 200 * 1024) return TN_EINVAL;
        gauge_kernel<<<1, 256, smem, c.st>>>(ga);
        TN_LAUNCHED();
    }
    GateArgs gt;                                                                          // a13
    Links L = make_links(c);
    for (int t = 0; t < c.nt; ++t)
        for (int g = 0; g < 4; ++g) {
            int e = L.link_of[t][g];
            gt.base[t][g] = L.is_out[t][g] ? c.fuP[e] : c.fuQ[e];
            gt.transposed[t][g] = L.is_out[t][g] ? 0 : 1;
            gt.maps[t][g] = c.cmaps[t][g];
            gt.W[t][g] = c.W[e];
            gt.K[t][g] = c.K[t][g];
        }
    gt.D = D;
    gate_kernel<<<4 * c.nt, 64, 0, c.st>>>(gt);
    TN_LAUNCHED();
    for (int t = 0; t < c.nt; ++t)
        TN_CUDA(cudaMemcpyAsync(c.A[t], c.A0[t], sizeof(double) * 2 * D * D * D * D, cudaMemcpyDeviceToDevice, c.st));
    if (F) {
        TN_CUDA(cudaMemcpyAsync(F, c.dscratch + 32, sizeof(double), cudaMemcpyDeviceToHost, c.st));
        TN_CUDA(cudaStreamSynchronize(c.st));
    }
    c.updated = false;
    c.have_gate = true;
    return TN_OK;
}

// n recycled steps with the window's gate: A <- (g A) x_legs K, max-abs normalised.
int recycle_advance(Ctx& c, int n_re)
{
    if (!c.have_gate) return TN_ESTATE;
    const int D = c.D;
    for (int r = 0; r < n_re; ++r)
        for (int t = 0; t < c.nt; ++t) {
            TN_TRY(apply_pepo(c, c.A[t], c.Theta[t]));
            size_t mk = c.ar.mark();
            double* b0 = c.ar.take((size_t)2 * c.kD * c.kD * c.kD * c.kD);
            double* b1 = c.ar.take((size_t)2 * c.kD * c.kD * c.kD * c.kD);
            if (!b0 || !b1) return TN_ENOMEM;
            int dims[5] = {2, c.kD, c.kD, c.kD, c.kD};
            const double* src = c.Theta[t];
            double* bufs[2] = {b0, b1};
            for (int g = 0; g < 4; ++g) {
                double* dst = (g == 3) ? c.A[t] : bufs[g & 1];
                TN_TRY(leg_mul(c, src, dst, dims, 1 + g, c.K[t][g], D));
                dims[1 + g] = D;
                src = dst;
            }
            TN_TRY(normalize_maxabs(c.st, c.A[t], 2LL * D * D * D * D, 1, 0));
            c.ar.release(mk);
        }
    bool ok = true;
    TN_TRY(state_finite(c, c.A, &ok));
    return ok ? TN_OK : TN_ENUMERIC;
}

int recycle(Ctx& c, int n_re, double* F)
{
    TN_TRY(recycle_build(c, F));
    return recycle_advance(c, n_re);
}

// change[0] = max over link types of ||N4 - ref||_F / ||ref||_F (one block per link)
__global__ void env_change_kernel(const double* __restrict__ N4, const double* __restrict__ ref, int n4, int nl,
                                  double* __restrict__ change)
{
    __shared__ double red[32];
    __shared__ double part[MAXL];
    for (int e = 0; e < nl; ++e) {
        double dn = 0.0, rn = 0.0;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) {
            const double r = ref[(size_t)e * n4 + i], d = N4[(size_t)e * n4 + i] - r;
            dn = fma(d, d, dn); rn = fma(r, r, rn);
        }
        dn = block_sum(dn, red);
        rn = block_sum(rn, red);
        if (threadIdx.x == 0) part[e] = rn > 0.0 ? sqrt(dn / rn) : (dn > 0.0 ? INFINITY : 0.0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int e = 0; e < nl; ++e) m = fmax(m, part[e]);
        change[0] = m;
    }
}

int env_change(Ctx& c, double* out)
{
    const int k = c.kD, n4 = k * k * k * k;
    env_change_kernel<<<1, 256, 0, c.st>>>(c.N4[0], c.N4ref, n4, c.nl, c.dscratch + 40);
    TN_LAUNCHED();
    TN_CUDA(cudaMemcpyAsync(out, c.dscratch + 40, sizeof(double), cudaMemcpyDeviceToHost, c.st));
    TN_CUDA(cudaStreamSynchronize(c.st));
    return TN_OK;
}

// RDMs and observables (a14): environment of the state's own double layers.
int measure(Ctx& c, tn_observables* obs)
{
    const int chi = c.chi, L = c.leg, D = c.D;
    if (L != D * D) return TN_ESTATE;
    size_t mk = c.ar.mark();
    double* rho1 = c.ar.take(4 * MAXT);
    double* rho2 = c.ar.take(16 * MAXL);
    double* res = c.ar.take(16);
    double* t1 = c.ar.take((size_t)chi * chi * L);
    double* top = c.ar.take((size_t)chi * chi * L);
    double* bot = c.ar.take((size_t)chi * chi * L);
    double* R1 = c.ar.take((size_t)chi * chi * L * L);
    double* R2 = c.ar.take((size_t)chi * chi * L * L);
    double* R3 = c.ar.take((size_t)L * L * L * L);
    double* K1 = c.ar.take((size_t)2 * D * D * D * D);
    double* Ar = c.ar.take((size_t)2 * D * D * D * D);
    double* Aq = c.ar.take((size_t)2 * D * D * D * D);
    double* X3 = c.ar.take((size_t)chi * chi * D * D * 2 * D * D);
    double* X4 = c.ar.take((size_t)chi * chi * D * D * D * D * 4);
    double* EL = c.ar.take((size_t)chi * chi * D * D * 4);
    double* ER = c.ar.take((size_t)chi * chi * D * D * 4);
    if (!rho1 || !rho2 || !res || !t1 || !top || !bot || !R1 || !R2 || !R3 || !K1 || !Ar || !Aq || !X3 || !X4 || !EL || !ER)
        return TN_ENOMEM;
    Frame f = c.frame0();
    const int tpos[2][2] = {{0, 0}, {1, 0}};
    auto Cm = [&](Env& e, int kk) { return dt(e.C[kk], {chi, chi}); };
    auto Tm = [&](Env& e, int kk) { return dt(e.T[kk], {chi, chi, L}); };
    for (int t = 0; t < c.nt; ++t) {                 // one-site RDM of each tensor
        Env& e = f.e(tpos[t][0], tpos[t][1]);
        TN_TRY(contract(c.st, c.ar, "ia,abm->ibm", Cm(e, 0), Tm(e, 0), dt(t1, {chi, chi, L})));
        TN_TRY(contract(c.st, c.ar, "ibm,bc->icm", dt(t1, {chi, chi, L}), Cm(e, 1), dt(top, {chi, chi, L})));
        TN_TRY(contract(c.st, c.ar, "de,efx->dfx", Cm(e, 2), Tm(e, 2), dt(t1, {chi, chi, L})));
        TN_TRY(contract(c.st, c.ar, "dfx,fj->djx", dt(t1, {chi, chi, L}), Cm(e, 3), dt(bot, {chi, chi, L})));
        // R3[(U u), (R r), (D d), (L l)] = top.T2 (R1) against bot.T4 (R2): the two halves
        // meet over (i, d), so no chi^2 L^3 intermediate is formed
        TN_TRY(contract(c.st, c.ar, "icm,cdn->imdn", dt(top, {chi, chi, L}), Tm(e, 1), dt(R1, {chi, L, chi, L})));
        TN_TRY(contract(c.st, c.ar, "djx,jil->dxil", dt(bot, {chi, chi, L}), Tm(e, 3), dt(R2, {chi, L, chi, L})));
        TN_TRY(contract(c.st, c.ar, "imdn,dxil->mnxl", dt(R1, {chi, L, chi, L}), dt(R2, {chi, L, chi, L}), dt(R3, {L, L, L, L})));
        TN_TRY(contract(c.st, c.ar, "UuRrDdLl,sLRDU->urdls", dt(R3, {D, D, D, D, D, D, D, D}), dt(c.A[t], {2, D, D, D, D}),
                        dt(K1, {D, D, D, D, 2})));
        TN_TRY(contract(c.st, c.ar, "urdls,tlrdu->st", dt(K1, {D, D, D, D, 2}), dt(c.A[t], {2, D, D, D, D}), dt(rho1 + 4 * t, {2, 2})));
    }
    Links lk = make_links(c);
    Frame fr = f.rotated();
    for (int e = 0; e < c.nl; ++e) {                 // two-site RDM of each link type
        const int t = lk.out_t[e], tq = lk.in_t[e];
        const bool vertical = e >= c.nt;
        int xp = tpos[t][0], yp = tpos[t][1];
        Frame* fp = &f;
        const double* Ap = c.A[t];
        const double* Aqp = c.A[tq];
        if (vertical) {
            const int dd[5] = {2, D, D, D, D}, rot5[5] = {0, 4, 3, 1, 2};
            TN_TRY(permute(c.st, c.A[t], Ar, 5, dd, rot5));
            TN_TRY(permute(c.st, c.A[tq], Aq, 5, dd, rot5));
            Ap = Ar; Aqp = Aq;
            int xr = ((yp % f.Ly) + f.Ly) % f.Ly, yr = ((-xp) % f.Lx + f.Lx) % f.Lx;
            xp = xr; yp = yr;
            fp = &fr;
        }
        Env& ep = fp->e(xp, yp);
        Env& eq = fp->e(xp + 1, yp);
        TN_TRY(contract(c.st, c.ar, "ia,aom->iom", Cm(ep, 0), Tm(ep, 0), dt(t1, {chi, chi, L})));
        TN_TRY(contract(c.st, c.ar, "iom,jin->omjn", dt(t1, {chi, chi, L}), Tm(ep, 3), dt(R1, {chi, L, chi, L})));
        TN_TRY(contract(c.st, c.ar, "oUujLl,sLRDU->oujlsRD", dt(R1, {chi, D, D, chi, D, D}), dt((double*)Ap, {2, D, D, D, D}),
                        dt(X3, {chi, D, chi, D, 2, D, D})));
        TN_TRY(contract(c.st, c.ar, "oujlsRD,tlrdu->ojRDrdst", dt(X3, {chi, D, chi, D, 2, D, D}), dt((double*)Ap, {2, D, D, D, D}),
                        dt(X4, {chi, chi, D, D, D, D, 2, 2})));
        TN_TRY(contract(c.st, c.ar, "kj,nkm->jnm", Cm(ep, 3), Tm(ep, 2), dt(top, {chi, chi, L})));
        TN_TRY(contract(c.st, c.ar, "ojRDrdst,jnDd->onRrst", dt(X4, {chi, chi, D, D, D, D, 2, 2}), dt(top, {chi, chi, D, D}),
                        dt(EL, {chi, chi, D, D, 2, 2})));
        TN_TRY(contract(c.st, c.ar, "oam,ac->ocm", Tm(eq, 0), Cm(eq, 1), dt(t1, {chi, chi, L})));
        TN_TRY(contract(c.st, c.ar, "ocm,ctn->omtn", dt(t1, {chi, chi, L}), Tm(eq, 1), dt(R1, {chi, L, chi, L})));
        TN_TRY(contract(c.st, c.ar, "oUutRr,sLRDU->outrsLD", dt(R1, {chi, D, D, chi, D, D}), dt((double*)Aqp, {2, D, D, D, D}),
                        dt(X3, {chi, D, chi, D, 2, D, D})));
        TN_TRY(contract(c.st, c.ar, "outrsLD,plrdu->otLDldsp", dt(X3, {chi, D, chi, D, 2, D, D}), dt((double*)Aqp, {2, D, D, D, D}),
                        dt(X4, {chi, chi, D, D, D, D, 2, 2})));
        TN_TRY(contract(c.st, c.ar, "te,enm->tnm", Cm(eq, 2), Tm(eq, 2), dt(bot, {chi, chi, L})));
        TN_TRY(contract(c.st, c.ar, "otLDldsp,tnDd->onLlsp", dt(X4, {chi, chi, D, D, D, D, 2, 2}), dt(bot, {chi, chi, D, D}),
                        dt(ER, {chi, chi, D, D, 2, 2})));
        TN_TRY(contract(c.st, c.ar, "onABsp,onABtq->stpq", dt(EL, {chi, chi, D, D, 2, 2}), dt(ER, {chi, chi, D, D, 2, 2}),
                        dt(rho2 + 16 * e, {2, 2, 2, 2})));
    }
    expect_kernel<<<1, 32, 0, c.st>>>(rho1, c.nt, rho2, c.nl, c.J, c.h, res);
    TN_LAUNCHED();
    double hres[16];
    TN_CUDA(cudaMemcpyAsync(hres, res, sizeof(double) * 10, cudaMemcpyDeviceToHost, c.st));
    TN_CUDA(cudaStreamSynchronize(c.st));
    obs->e_site = hres[0];
    obs->e_link = hres[1];
    for (int t = 0; t < 2; ++t) { obs->mx[t] = t < c.nt ? hres[2 + t] : 0.0; obs->mz[t] = t < c.nt ? hres[4 + t] : 0.0; }
    for (int e = 0; e < 4; ++e) obs->zz[e] = e < c.nl ? hres[6 + e] : 0.0;
    c.ar.release(mk);
    return TN_OK;
}

}  // namespace tn
