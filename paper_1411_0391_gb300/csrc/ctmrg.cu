// CTMRG environment of the double-layer network (Sec. VI.B item 1, Fig. 21a),
// rows a2-a6 of the hot path.
//
// Reading of the cited CTMRG (the paper gives no moves): directional moves
// left, up, right, down; up/right/down are the left move in the frame rotated
// counter-clockwise 1, 2, 3 times (a relabelling of pointers, no data moves).
// A left move absorbs the columns x = 0..Lx-1 in turn; for every cut (y|y+1)
// of a column the four enlarged corners give R_u = Q_UL Q_UR, R_d = Q_LR Q_LL
// and the loop rho = R_d R_u = U S V^T (top chi, sign rule), from which
//   P_up = R_d^T U S^{-1/2},  P_lo = R_u V S^{-1/2}
// (S^{-1/2} = 0 below 1e-12 s_1).  The new C1, T4, C4 of column x+1 are
//   C1' = P_up(y-1|y)^T (C1 T1),  T4' = P_up(y|y+1)^T (T4 a) P_lo(y-1|y),
//   C4' = (C4 T3) P_lo(y|y+1),
// each divided by its largest |entry|.  All environment tensors keep the fixed
// shapes chi x chi and chi x chi x leg; unused directions are zeros.
#include <algorithm>
#include <cmath>
#include <thread>
#include "ctx.cuh"

namespace tn {

static const int CORNER_LEGS[4][4] = {
    {0, 3, 2, 1},   // UL: a.l joins T4, a.u joins T1, rows a.d, cols a.r
    {3, 1, 0, 2},   // UR: a.u joins T1, a.r joins T2, rows a.l, cols a.d
    {1, 2, 3, 0},   // LR: a.r joins T2, a.d joins T3, rows a.u, cols a.l
    {2, 0, 1, 3},   // LL: a.d joins T3, a.l joins T4, rows a.r, cols a.u
};

Frame Frame::rotated() const
{
    Frame f;
    f.Lx = Ly; f.Ly = Lx; f.rot = (rot + 1) & 3;
    for (int y2 = 0; y2 < f.Ly; ++y2)
        for (int x2 = 0; x2 < f.Lx; ++x2) f.pat[y2][x2] = tid(-y2, x2);
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            const Env& o = env[y * Lx + x];
            int x2 = ((y % Ly) + Ly) % Ly, y2 = ((-x) % Lx + Lx) % Lx;
            Env& n = f.env[y2 * f.Lx + x2];
            for (int k = 0; k < 4; ++k) { n.C[k] = o.C[(k + 1) & 3]; n.T[k] = o.T[(k + 1) & 3]; }
        }
    return f;
}

Frame Ctx::frame0()
{
    Frame f;
    f.Lx = Lx; f.Ly = Ly; f.rot = 0;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) { f.pat[y][x] = pat[y][x]; f.env[y * Lx + x] = env0[y * Lx + x]; }
    return f;
}

int ctx_build_network_views(Ctx& c)
{
    const int L = c.leg;
    const int dims[4] = {L, L, L, L};
    const int rot[4] = {3, 2, 0, 1};          // a'[L,R,D,U] = a[D',U',R',L'] (counter-clockwise)
    for (int t = 0; t < c.nt; ++t) {
        for (int r = 1; r < 4; ++r) TN_TRY(permute(c.st, c.a[r - 1][t], c.a[r][t], 4, dims, rot));
        for (int r = 0; r < 4; ++r) {
            for (int k = 0; k < 4; ++k) TN_TRY(permute(c.st, c.a[r][t], c.ab[r][t][k], 4, dims, CORNER_LEGS[k]));
            const int p4[4] = {2, 0, 1, 3};   // [d, l, r, u]
            TN_TRY(permute(c.st, c.a[r][t], c.aT4[r][t], 4, dims, p4));
        }
    }
    return TN_OK;
}

__global__ void init_env_kernel(double* env, int nsites, int chi, int leg, const double* boundary)
{
    const size_t per = 4 * (size_t)chi * chi + 4 * (size_t)chi * chi * leg;
    for (int s = blockIdx.x; s < nsites; s += gridDim.x) {
        double* e = env + s * per;
        for (int k = 0; k < 4; ++k) if (threadIdx.x == 0) e[(size_t)k * chi * chi] = 1.0;
        double* T = e + 4 * (size_t)chi * chi;
        for (int k = 0; k < 4; ++k)
            for (int m = threadIdx.x; m < leg; m += blockDim.x) T[(size_t)k * chi * chi * leg + m] = boundary[m];
    }
}

int ctx_reset_env(Ctx& c)
{
    TN_TRY(fill(c.st, c.envbuf, (long long)c.env_size(), 0.0));
    init_env_kernel<<<c.nsites, 128, 0, c.st>>>(c.envbuf, c.nsites, c.chi, c.leg, c.boundary);
    TN_LAUNCHED();
    for (int r = 0; r < 4; ++r) for (int x = 0; x < 4; ++x) for (int y = 0; y < 4; ++y) c.warm_ok[r][x][y] = false;
    c.prev_spectra.clear();
    c.split_ready = false;
    c.fp64_moves = 0;
    return TN_OK;
}

// P[:, j] *= (s_j >= cut * s_0) ? 1/sqrt(s_j) : 0
__global__ void scale_cols_invsqrt_kernel(double* P, int rows, int cols, const double* s, double cut)
{
    const double s0 = s[0];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)rows * cols;
         e += (long long)gridDim.x * blockDim.x) {
        int j = (int)(e % cols);
        double sj = s[j];
        P[e] *= (s0 > 0.0 && sj >= cut * s0) ? rsqrt(sj) : 0.0;
    }
}

static int scale_cols_invsqrt(cudaStream_t st, double* P, int rows, int cols, const double* s, double cut)
{
    long long total = (long long)rows * cols;
    int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 8);
    scale_cols_invsqrt_kernel<<<blocks, 256, 0, st>>>(P, rows, cols, s, cut);
    TN_LAUNCHED();
    return TN_OK;
}

// Enlarged corner of type k at a site: C[k] with edges Ta = T[k] (after) and
// Tb = T[k-1] (before), as the N x N matrix [(Tb.in, row), (Ta.out, col)].
static int enlarged_corner(Ctx& c, cudaStream_t st, Arena& ar, const Env& e, int k, const double* ab, double* Q)
{
    const int chi = c.chi, L = c.leg;
    size_t mk = ar.mark();
    double* X = ar.take((size_t)chi * chi * L);
    double* Y = ar.take((size_t)chi * chi * L * L);
    if (!X || !Y) return TN_ENOMEM;
    const double* C = e.C[k];
    const double* Ta = e.T[k];
    const double* Tb = e.T[(k + 3) & 3];
    const int kd = c.kind();
    // X[o, j, n] = C[o, a] Ta[a, j, n]
    TN_TRY(gemm_any(st, ar, kd, false, false, chi, chi * L, chi, 1.0, C, chi, Ta, chi * L, 0.0, X, chi * L));
    // Y[i, m, j, n] = Tb[i, o, m] X[o, j, n]
    TN_TRY(contract(st, ar, "iom,ojn->imjn", dt((double*)Tb, {chi, chi, L}), dt(X, {chi, chi, L}),
                    dt(Y, {chi, L, chi, L}), 1.0, 0.0, kd));
    // Q[i, r, j, q] = Y[i, m, j, n] ab[m, n, r, q]
    TN_TRY(contract(st, ar, "imjn,mnrq->irjq", dt(Y, {chi, L, chi, L}), dt((double*)ab, {L, L, L, L}),
                    dt(Q, {chi, L, chi, L}), 1.0, 0.0, kd));
    ar.release(mk);
    return TN_OK;
}

// Projectors of the cut (y | y+1) of column x in frame f, on stream st with the
// scratch arena ar (the cuts of a column are independent: each may run on its
// own stream and arena).  stats: the projector SVD's subspace iterations.
static int cut_projectors(Ctx& c, Frame& f, int x, int y, double* Pup, double* Plo, cudaStream_t st, Arena& ar,
                          TsvdStats& stats)
{
    const int N = c.N(), chi = c.chi;
    size_t mk = ar.mark();
    double* Q[4];
    for (int k = 0; k < 4; ++k) if (!(Q[k] = ar.take((size_t)N * N))) return TN_ENOMEM;
    const int xs[4] = {x, x + 1, x + 1, x};
    const int ys[4] = {y, y, y + 1, y + 1};
    for (int k = 0; k < 4; ++k) {
        int t = f.tid(xs[k], ys[k]);
        TN_TRY(enlarged_corner(c, st, ar, f.e(xs[k], ys[k]), k, c.ab[f.rot][t][k], Q[k]));
    }
    double* Ru = ar.take((size_t)N * N);
    double* Rd = ar.take((size_t)N * N);
    double* rho = ar.take((size_t)N * N);
    double* U = ar.take((size_t)N * chi);
    double* S = ar.take(chi);
    if (!Ru || !Rd || !rho || !U || !S) return TN_ENOMEM;
    const int kd = c.kind();
    TN_TRY(gemm_any(st, ar, kd, false, false, N, N, N, 1.0, Q[0], N, Q[1], N, 0.0, Ru, N));
    TN_TRY(gemm_any(st, ar, kd, false, false, N, N, N, 1.0, Q[2], N, Q[3], N, 0.0, Rd, N));
    TN_TRY(gemm_any(st, ar, kd, false, false, N, N, N, 1.0, Rd, N, Ru, N, 0.0, rho, N));
    const int xx = ((x % f.Lx) + f.Lx) % f.Lx, yy = ((y % f.Ly) + f.Ly) % f.Ly;
    double* Vw = c.warmV[f.rot][xx][yy];
    // V goes straight into the warm-start slot of this cut
    // the projector SVD runs in FP64 in every mode; its products with rho run on the SIMT
    // pipe or, in the slice forms, as FP64-accurate 7-slice tensor-core products
    int s = truncated_svd(st, ar, rho, N, chi, U, S, Vw, c.warm_ok[f.rot][xx][yy] ? Vw : nullptr, &stats,
                          c.svd_kind(), c.svd_tol());
    if (s != TN_OK && s != TN_ENOCONV) return s;
    c.warm_ok[f.rot][xx][yy] = true;
    // P_up = R_d^T U S^{-1/2}, P_lo = R_u V S^{-1/2}
    TN_TRY(gemm_any(st, ar, kd, true, false, N, chi, N, 1.0, Rd, N, U, chi, 0.0, Pup, chi));
    TN_TRY(gemm_any(st, ar, kd, false, false, N, chi, N, 1.0, Ru, N, Vw, chi, 0.0, Plo, chi));
    TN_TRY(scale_cols_invsqrt(st, Pup, N, chi, S, c.proj_cut()));
    TN_TRY(scale_cols_invsqrt(st, Plo, N, chi, S, c.proj_cut()));
    ar.release(mk);
    return TN_OK;
}

// New C1, T4, C4 for column x+1 from the environment of (x, y).
static int renormalize(Ctx& c, Frame& f, int x, int y, const double* pu_above, const double* pl_above,
                       const double* pu, const double* pl, double* C1n, double* T4n, double* C4n)
{
    const int chi = c.chi, L = c.leg;
    const int t = f.tid(x, y);
    Env& e = f.e(x, y);
    size_t mk = c.ar.mark();
    double* CT = c.ar.take((size_t)chi * chi * L);
    double* X1 = c.ar.take((size_t)chi * chi * L * L);
    double* X2 = c.ar.take((size_t)chi * chi * L * L);
    double* TC = c.ar.take((size_t)chi * chi * L);
    if (!CT || !X1 || !X2 || !TC) return TN_ENOMEM;
    const int kd = c.kind();
    // C1'[a, o] = P_up(y-1|y)[i, m, a] C1[i, c] T1[c, o, m]
    TN_TRY(gemm_any(c.st, c.ar, kd, false, false, chi, chi * L, chi, 1.0, e.C[0], chi, e.T[0], chi * L, 0.0, CT, chi * L));
    TN_TRY(contract(c.st, c.ar, "ima,iom->ao", dt((double*)pu_above, {chi, L, chi}), dt(CT, {chi, chi, L}),
                    dt(C1n, {chi, chi}), 1.0, 0.0, kd));
    // T4'[a, b, r] = P_up(y|y+1)[i, s, a] T4[i, j, m] a[m, r, s, t] P_lo(y-1|y)[j, t, b]
    TN_TRY(contract(c.st, c.ar, "isa,ijm->sajm", dt((double*)pu, {chi, L, chi}), dt(e.T[3], {chi, chi, L}),
                    dt(X1, {L, chi, chi, L}), 1.0, 0.0, kd));
    TN_TRY(contract(c.st, c.ar, "sajm,smrt->ajrt", dt(X1, {L, chi, chi, L}), dt(c.aT4[f.rot][t], {L, L, L, L}),
                    dt(X2, {chi, chi, L, L}), 1.0, 0.0, kd));
    TN_TRY(contract(c.st, c.ar, "ajrt,jtb->abr", dt(X2, {chi, chi, L, L}), dt((double*)pl_above, {chi, L, chi}),
                    dt(T4n, {chi, chi, L}), 1.0, 0.0, kd));
    // C4'[i, a] = C4[c, q] T3[i, c, m] P_lo(y|y+1)[q, m, a]
    TN_TRY(contract(c.st, c.ar, "icm,cq->iqm", dt(e.T[2], {chi, chi, L}), dt(e.C[3], {chi, chi}),
                    dt(TC, {chi, chi, L}), 1.0, 0.0, kd));
    TN_TRY(contract(c.st, c.ar, "iqm,qma->ia", dt(TC, {chi, chi, L}), dt((double*)pl, {chi, L, chi}),
                    dt(C4n, {chi, chi}), 1.0, 0.0, kd));
    TN_TRY(normalize_maxabs(c.st, C1n, (long long)chi * chi, 1, 0));
    TN_TRY(normalize_maxabs(c.st, T4n, (long long)chi * chi * L, 1, 0));
    TN_TRY(normalize_maxabs(c.st, C4n, (long long)chi * chi, 1, 0));
    c.ar.release(mk);
    return TN_OK;
}

// Projectors of every cut of column x.  The cuts are independent: with more than
// one, each runs on its own stream (ordered after the context stream by an
// event, joined back by events) and its own slice of the scratch arena, driven
// by its own host thread, so that the latency-bound factorisations of the
// projector SVDs (one SM each) and the host's waits on their convergence tests
// overlap.
static int column_projectors(Ctx& c, Frame& f, int x)
{
    const int ny = f.Ly;
    TsvdStats stats[MAXS];
    if (ny == 1 || !c.cut_st[0]) {
        for (int y = 0; y < ny; ++y) TN_TRY(cut_projectors(c, f, x, y, c.Pup[y], c.Plo[y], c.st, c.ar, stats[y]));
    } else {
        const size_t base = c.ar.mark();
        const size_t share = ((c.ar.cap - base) / ny) & ~size_t(255);
        Arena sub[MAXS];
        for (int y = 0; y < ny; ++y) {
            sub[y].base = c.ar.base + base + (size_t)y * share;
            sub[y].cap = share;
        }
        TN_CUDA(cudaEventRecord(c.ev_fork, c.st));
        for (int y = 0; y < ny; ++y) TN_CUDA(cudaStreamWaitEvent(c.cut_st[y], c.ev_fork, 0));
        int status[MAXS];
        int dev = 0;
        TN_CUDA(cudaGetDevice(&dev));
        std::vector<std::thread> workers;
        for (int y = 1; y < ny; ++y)
            workers.emplace_back([&, y]() {
                cudaSetDevice(dev);
                status[y] = cut_projectors(c, f, x, y, c.Pup[y], c.Plo[y], c.cut_st[y], sub[y], stats[y]);
            });
        status[0] = cut_projectors(c, f, x, 0, c.Pup[0], c.Plo[0], c.cut_st[0], sub[0], stats[0]);
        for (auto& w : workers) w.join();
        for (int y = 0; y < ny; ++y) {
            TN_CUDA(cudaEventRecord(c.ev_join[y], c.cut_st[y]));
            TN_CUDA(cudaStreamWaitEvent(c.st, c.ev_join[y], 0));
        }
        for (int y = 0; y < ny; ++y) TN_TRY(status[y]);
    }
    for (int y = 0; y < ny; ++y) {
        c.svd_calls += 1;
        c.svd_iterations += stats[y].iterations;
    }
    return TN_OK;
}

int ctmrg_move(Ctx& c, Frame& f)
{
    const int chi = c.chi, L = c.leg, N = c.N();
    for (int x = 0; x < f.Lx; ++x) {
        TN_TRY(column_projectors(c, f, x));
        size_t mk = c.ar.mark();
        double* nC1[4]; double* nT4[4]; double* nC4[4];
        for (int y = 0; y < f.Ly; ++y) {
            nC1[y] = c.ar.take((size_t)chi * chi);
            nT4[y] = c.ar.take((size_t)chi * chi * L);
            nC4[y] = c.ar.take((size_t)chi * chi);
            if (!nC1[y] || !nT4[y] || !nC4[y]) return TN_ENOMEM;
        }
        for (int y = 0; y < f.Ly; ++y) {
            int ya = (y - 1 + f.Ly) % f.Ly;
            TN_TRY(renormalize(c, f, x, y, c.Pup[ya], c.Plo[ya], c.Pup[y], c.Plo[y], nC1[y], nT4[y], nC4[y]));
        }
        for (int y = 0; y < f.Ly; ++y) {
            Env& tgt = f.e(x + 1, y);
            TN_CUDA(cudaMemcpyAsync(tgt.C[0], nC1[y], sizeof(double) * chi * chi, cudaMemcpyDeviceToDevice, c.st));
            TN_CUDA(cudaMemcpyAsync(tgt.T[3], nT4[y], sizeof(double) * chi * chi * L, cudaMemcpyDeviceToDevice, c.st));
            TN_CUDA(cudaMemcpyAsync(tgt.C[3], nC4[y], sizeof(double) * chi * chi, cudaMemcpyDeviceToDevice, c.st));
        }
        c.ar.release(mk);
        (void)N;
    }
    ++c.ctm_moves;
    if (!c.split_ready && ++c.fp64_moves >= 32) c.split_ready = true;
    return TN_OK;
}

int ctmrg_moves(Ctx& c, int n)
{
    Frame f = c.frame0();
    for (int i = 0; i < n; ++i) {
        TN_TRY(ctmrg_move(c, f));
        f = f.rotated();
    }
    return TN_OK;
}

int corner_spectra(Ctx& c, std::vector<double>& out)
{
    const int chi = c.chi, nb = 4 * c.nsites;
    size_t mk = c.ar.mark();
    double* Cs = c.ar.take((size_t)nb * chi * chi);
    double* U = c.ar.take((size_t)nb * chi * chi);
    double* S = c.ar.take((size_t)nb * chi);
    double* V = c.ar.take((size_t)nb * chi * chi);
    if (!Cs || !U || !S || !V) return TN_ENOMEM;
    for (int s = 0; s < c.nsites; ++s)
        TN_CUDA(cudaMemcpyAsync(Cs + (size_t)s * 4 * chi * chi, c.env0[s].C[0], sizeof(double) * 4 * chi * chi,
                                cudaMemcpyDeviceToDevice, c.st));
    TN_TRY(svd_small(c.st, Cs, chi, chi, nb, U, S, V));
    out.resize((size_t)nb * chi);
    TN_CUDA(cudaMemcpyAsync(out.data(), S, sizeof(double) * nb * chi, cudaMemcpyDeviceToHost, c.st));
    TN_CUDA(cudaStreamSynchronize(c.st));
    for (int b = 0; b < nb; ++b) {
        double tot = 0.0;
        for (int i = 0; i < chi; ++i) tot += out[(size_t)b * chi + i];
        if (tot > 0.0) for (int i = 0; i < chi; ++i) out[(size_t)b * chi + i] /= tot;
    }
    c.ar.release(mk);
    return TN_OK;
}

int ctmrg_iterations(Ctx& c, double tol, int max_iter, tn_ctm_report* rep)
{
    std::vector<double> cur;
    const long long calls0 = c.svd_calls, iters0 = c.svd_iterations;
    if (c.prev_spectra.empty()) TN_TRY(corner_spectra(c, c.prev_spectra));
    double delta = INFINITY;
    int it = 0;
    bool conv = false;
    for (it = 1; it <= max_iter; ++it) {
        TN_TRY(ctmrg_moves(c, 4));
        TN_TRY(corner_spectra(c, cur));
        delta = 0.0;
        const int chi = c.chi;
        for (int b = 0; b < 4 * c.nsites; ++b) {
            double acc = 0.0;
            for (int i = 0; i < chi; ++i) {
                double d = cur[(size_t)b * chi + i] - c.prev_spectra[(size_t)b * chi + i];
                acc += d * d;
            }
            delta = std::max(delta, std::sqrt(acc));
        }
        c.prev_spectra = cur;
        if (delta <= 1e-4) c.split_ready = true;
        if (!std::isfinite(delta)) {
            if (rep) { rep->iterations = it; rep->converged = 0; rep->delta = delta; rep->svd_calls = 0; rep->svd_iterations = 0; }
            return TN_ENUMERIC;
        }
        if (delta < tol) { conv = true; break; }
    }
    if (it > max_iter) it = max_iter;
    if (rep) {
        rep->iterations = it; rep->converged = conv ? 1 : 0; rep->delta = delta;
        rep->svd_calls = (int)(c.svd_calls - calls0); rep->svd_iterations = (int)(c.svd_iterations - iters0);
    }
    return conv ? TN_OK : TN_ENOCONV;
}

int site_scalars(Ctx& c, int site, const double* d_a, double out[4])
{
    const int chi = c.chi, L = c.leg;
    Env& e = c.env0[site];
    const int x = site % c.Lx, y = site / c.Lx;
    const double* a = d_a ? d_a : c.a[0][c.pat[y][x]];
    size_t mk = c.ar.mark();
    double* t1 = c.ar.take((size_t)chi * chi * L);
    double* top = c.ar.take((size_t)chi * chi * L);
    double* bot = c.ar.take((size_t)chi * chi * L);
    double* R1 = c.ar.take((size_t)chi * chi * L * L);
    double* R2 = c.ar.take((size_t)chi * chi * L * L * L);
    double* R3 = c.ar.take((size_t)L * L * L * L);
    double* m1 = c.ar.take((size_t)chi * chi);
    double* m2 = c.ar.take((size_t)chi * chi);
    double* sc = c.ar.take(4);
    if (!t1 || !top || !bot || !R1 || !R2 || !R3 || !m1 || !m2 || !sc) return TN_ENOMEM;
    auto Cm = [&](int k) { return dt(e.C[k], {chi, chi}); };
    auto Tm = [&](int k) { return dt(e.T[k], {chi, chi, L}); };
    DT s0 = dt(sc, {}), s1 = dt(sc + 1, {}), s2 = dt(sc + 2, {}), s3 = dt(sc + 3, {});
    TN_TRY(contract(c.st, c.ar, "ia,abm->ibm", Cm(0), Tm(0), dt(t1, {chi, chi, L})));
    TN_TRY(contract(c.st, c.ar, "ibm,bc->icm", dt(t1, {chi, chi, L}), Cm(1), dt(top, {chi, chi, L})));
    TN_TRY(contract(c.st, c.ar, "de,efx->dfx", Cm(2), Tm(2), dt(t1, {chi, chi, L})));
    TN_TRY(contract(c.st, c.ar, "dfx,fj->djx", dt(t1, {chi, chi, L}), Cm(3), dt(bot, {chi, chi, L})));
    TN_TRY(contract(c.st, c.ar, "icu,cdr->iudr", dt(top, {chi, chi, L}), Tm(1), dt(R1, {chi, L, chi, L})));
    TN_TRY(contract(c.st, c.ar, "iudr,djx->iurjx", dt(R1, {chi, L, chi, L}), dt(bot, {chi, chi, L}),
                    dt(R2, {chi, L, L, chi, L})));
    TN_TRY(contract(c.st, c.ar, "iurjx,jil->urxl", dt(R2, {chi, L, L, chi, L}), Tm(3), dt(R3, {L, L, L, L})));
    TN_TRY(contract(c.st, c.ar, "urxl,lrxu->", dt(R3, {L, L, L, L}), dt((double*)a, {L, L, L, L}), s0));
    TN_TRY(contract(c.st, c.ar, "ia,ab->ib", Cm(0), Cm(1), dt(m1, {chi, chi})));
    TN_TRY(contract(c.st, c.ar, "ib,bc->ic", dt(m1, {chi, chi}), Cm(2), dt(m2, {chi, chi})));
    TN_TRY(contract(c.st, c.ar, "ic,ci->", dt(m2, {chi, chi}), Cm(3), s1));
    TN_TRY(contract(c.st, c.ar, "icm,cim->", dt(top, {chi, chi, L}), dt(bot, {chi, chi, L}), s2));
    // Zv = C1 C2 T2 C3 C4 T4 with T2.m = T4.m
    TN_TRY(contract(c.st, c.ar, "ib,bcm->icm", dt(m1, {chi, chi}), Tm(1), dt(t1, {chi, chi, L})));
    TN_TRY(contract(c.st, c.ar, "cd,de->ce", Cm(2), Cm(3), dt(m2, {chi, chi})));
    TN_TRY(contract(c.st, c.ar, "ce,eim->cim", dt(m2, {chi, chi}), Tm(3), dt(top, {chi, chi, L})));
    TN_TRY(contract(c.st, c.ar, "icm,cim->", dt(t1, {chi, chi, L}), dt(top, {chi, chi, L}), s3));
    TN_CUDA(cudaMemcpyAsync(out, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    TN_CUDA(cudaStreamSynchronize(c.st));
    c.ar.release(mk);
    return TN_OK;
}

}  // namespace tn
