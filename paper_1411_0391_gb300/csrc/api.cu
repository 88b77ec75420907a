// Exported C ABI of libtnite (declared in include/tnite.h): argument checks,
// the device-workspace plan of a context, host<->device copies and the
// evolution driver.  All device memory is carved from the caller's workspace.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <atomic>
#include <thread>
#include "ctx.cuh"

namespace tn {

static thread_local cudaError_t g_last_cuda = cudaSuccess;

}  // namespace tn

void tn_last_cuda_error(cudaError_t e) { tn::g_last_cuda = e; }

static std::atomic<unsigned long long> g_launches{0};
void tn_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace tn {

static bool valid_cfg(const tn_config* cfg)
{
    if (!cfg) return false;
    if (cfg->D < 1 || cfg->D > 6) return false;
    if (cfg->chi < 1 || cfg->chi > 96) return false;
    if (cfg->cell != TN_CELL_CHECKERBOARD && cfg->cell != TN_CELL_SINGLE) return false;
    if (cfg->precision < TN_F64 || cfg->precision > TN_F64S7) return false;
    return true;
}

// Carve every buffer of a context from the arena (counting or real pass).
static bool plan(Ctx& c)
{
    const int D = c.cfg.D, chi = c.cfg.chi, L = D * D, k = 2 * D;
    const size_t nA = 2 * (size_t)D * D * D * D, nTh = 2 * (size_t)k * k * k * k, nN = (size_t)k * k * k * k;
    const size_t N = (size_t)chi * L;
    Arena& ar = c.ar;
    bool ok = true;
    auto take = [&](size_t n) { double* p = ar.take(n); if (!ar.counting && !p) ok = false; return p; };
    for (int t = 0; t < MAXT; ++t) {
        c.A[t] = take(nA); c.Ac[t] = take(nA); c.A0[t] = take(nA); c.A1[t] = take(nA); c.Asave[t] = take(nA);
        c.Theta[t] = take(nTh);
        for (int g = 0; g < 4; ++g) { c.cmaps[t][g] = take((size_t)D * D); c.K[t][g] = take((size_t)k * D); }
    }
    for (int e = 0; e < MAXL; ++e) {
        c.lam[e] = take(D);
        c.preP[e] = take((size_t)k * D); c.preQ[e] = take((size_t)k * D);
        c.fuP[e] = take((size_t)k * D); c.fuQ[e] = take((size_t)k * D);
        c.W[e] = take((size_t)D * D);
    }
    double* n4 = take(MAXL * nN);
    c.N4ref = take(MAXL * nN);
    for (int e = 0; e < MAXL; ++e) c.N4[e] = n4 ? n4 + e * nN : nullptr;
    c.g = take(64);
    const size_t nl4 = (size_t)L * L * L * L;
    for (int r = 0; r < 4; ++r)
        for (int t = 0; t < MAXT; ++t) {
            c.a[r][t] = take(nl4);
            c.aT4[r][t] = take(nl4);
            for (int q = 0; q < 4; ++q) c.ab[r][t][q] = take(nl4);
        }
    c.boundary = take(L);
    c.envbuf = take(c.env_size());
    for (int r = 0; r < 4; ++r)
        for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) c.warmV[r][x][y] = take(N * chi);
    for (int y = 0; y < 4; ++y) { c.Pup[y] = take(N * chi); c.Plo[y] = take(N * chi); }
    c.dscratch = take(64);
    c.scratch_base = ar.mark();
    // scratch for the largest step (CTMRG cut / bond environment / observables); the cuts of
    // a column run concurrently, each on its own share of the scratch
    const size_t cuts = c.cfg.cell == TN_CELL_CHECKERBOARD ? 2 : 1;
    const size_t scratch = cuts * (26 * N * N + 1200 * N + ((size_t)1 << 22));
    take(scratch);
    return ok;
}

static void setup_geometry(Ctx& c)
{
    c.D = c.cfg.D; c.chi = c.cfg.chi; c.kD = 2 * c.D; c.leg = c.D * c.D;
    if (c.cfg.cell == TN_CELL_CHECKERBOARD) {
        c.nt = 2; c.nl = 4; c.Lx = 2; c.Ly = 2;
        c.pat[0][0] = 0; c.pat[0][1] = 1; c.pat[1][0] = 1; c.pat[1][1] = 0;
    } else {
        c.nt = 1; c.nl = 2; c.Lx = 1; c.Ly = 1;
        c.pat[0][0] = 0;
    }
    c.nsites = c.Lx * c.Ly;
}

static void bind_env(Ctx& c)
{
    const size_t chi2 = (size_t)c.chi * c.chi, per = 4 * chi2 + 4 * chi2 * c.leg;
    for (int s = 0; s < c.nsites; ++s) {
        double* base = c.envbuf + s * per;
        for (int q = 0; q < 4; ++q) {
            c.env0[s].C[q] = base + q * chi2;
            c.env0[s].T[q] = base + 4 * chi2 + q * chi2 * c.leg;
        }
    }
}

static Ctx* C(void* p) { return reinterpret_cast<Ctx*>(p); }

}  // namespace tn

using namespace tn;

extern "C" {

unsigned long long tn_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

size_t tn_workspace_bytes(const tn_config* cfg)
{
    if (!valid_cfg(cfg)) return 0;
    Ctx c;
    c.cfg = *cfg;
    setup_geometry(c);
    c.ar.counting = true;
    plan(c);
    return c.ar.peak + 256;
}

int tn_create(void** out, const tn_config* cfg, void* ws, size_t bytes, void* stream)
{
    if (!out || !valid_cfg(cfg) || !ws) return TN_EINVAL;
    Ctx* c = new (std::nothrow) Ctx();
    if (!c) return TN_ENOMEM;
    c->cfg = *cfg;
    c->st = reinterpret_cast<cudaStream_t>(stream);
    setup_geometry(*c);
    uintptr_t base = (reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255);
    c->ar.base = reinterpret_cast<char*>(base);
    c->ar.cap = bytes - (base - reinterpret_cast<uintptr_t>(ws));
    if (bytes < tn_workspace_bytes(cfg) || !plan(*c)) { delete c; return TN_ENOMEM; }
    c->ar.release(c->scratch_base);
    bind_env(*c);
    // ket-bra identity boundary
    std::vector<double> b(c->leg, 0.0);
    for (int i = 0; i < c->D; ++i) b[i * c->D + i] = 1.0;
    if (cudaMemcpyAsync(c->boundary, b.data(), sizeof(double) * c->leg, cudaMemcpyHostToDevice, c->st) != cudaSuccess) {
        delete c; return TN_ECUDA;
    }
    if (c->Ly > 1) {            // streams and events of the concurrent cuts
        for (int y = 0; y < c->Ly; ++y) {
            if (cudaStreamCreateWithFlags(&c->cut_st[y], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&c->ev_join[y], cudaEventDisableTiming) != cudaSuccess) {
                delete c; return TN_ECUDA;
            }
        }
        if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) { delete c; return TN_ECUDA; }
    }
    int s = ctx_reset_env(*c);
    if (s != TN_OK) { delete c; return s; }
    if (cudaStreamSynchronize(c->st) != cudaSuccess) { delete c; return TN_ECUDA; }
    *out = c;
    return TN_OK;
}

void tn_destroy(void* ctx) { delete C(ctx); }

const char* tn_strerror(int s)
{
    switch (s) {
        case TN_OK: return "ok";
        case TN_EINVAL: return "invalid argument";
        case TN_ENOMEM: return "device workspace too small";
        case TN_ECUDA: return cudaGetErrorString(tn::g_last_cuda);
        case TN_ENOCONV: return "iteration cap reached (results written)";
        case TN_ENUMERIC: return "NaN or Inf encountered";
        case TN_ESTATE: return "call out of order (state, time step or environment missing)";
        case TN_ESCRATCH: return "problem larger than the fixed scratch of the allocation-free entry point";
        case TN_ETIMEOUT: return "a bounded device-side wait expired in a tensor-core kernel";
        case TN_EUNSTABLE: return "recycling judged unstable in some window; those steps were redone without recycling (results written)";
        default: return "unknown status";
    }
}

int tn_set_hamiltonian(void* ctx, double J, double h)
{
    if (!ctx || !(J > 0.0) || !std::isfinite(h)) return TN_EINVAL;
    C(ctx)->J = J; C(ctx)->h = h;
    C(ctx)->have_gate = false;            // the gate of a recycling window belongs to the old g
    if (C(ctx)->tau > 0.0) return build_pepo(*C(ctx));
    return TN_OK;
}

int tn_set_time_step(void* ctx, double tau)
{
    if (!ctx || !(tau > 0.0) || !std::isfinite(tau)) return TN_EINVAL;
    C(ctx)->tau = tau;
    C(ctx)->have_gate = false;
    return build_pepo(*C(ctx));
}

int tn_set_state(void* ctx, const double* host, size_t n)
{
    if (!ctx || !host) return TN_EINVAL;
    Ctx& c = *C(ctx);
    const size_t per = 2 * (size_t)c.D * c.D * c.D * c.D;
    if (n != per * c.nt) return TN_EINVAL;
    for (int t = 0; t < c.nt; ++t)
        TN_CUDA(cudaMemcpyAsync(c.A[t], host + t * per, per * sizeof(double), cudaMemcpyHostToDevice, c.st));
    TN_CUDA(cudaStreamSynchronize(c.st));
    c.have_state = true;
    c.have_gate = false;
    return TN_OK;
}

int tn_get_state(void* ctx, double* host, size_t n)
{
    if (!ctx || !host) return TN_EINVAL;
    Ctx& c = *C(ctx);
    const size_t per = 2 * (size_t)c.D * c.D * c.D * c.D;
    if (n != per * c.nt) return TN_EINVAL;
    for (int t = 0; t < c.nt; ++t)
        TN_CUDA(cudaMemcpyAsync(host + t * per, c.A[t], per * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    TN_CUDA(cudaStreamSynchronize(c.st));
    return TN_OK;
}

int tn_build_double_layer(void* ctx)
{
    if (!ctx) return TN_EINVAL;
    Ctx& c = *C(ctx);
    if (!c.have_state) return TN_ESTATE;
    if (c.leg != c.D * c.D) return TN_ESTATE;
    TN_TRY(build_double_layers(c, c.A, c.D));
    c.have_network = true;
    TN_CUDA(cudaStreamSynchronize(c.st));
    return TN_OK;
}

int tn_set_network(void* ctx, const double* a_host, int leg_dim, const double* boundary)
{
    if (!ctx || !a_host || leg_dim < 1) return TN_EINVAL;
    Ctx& c = *C(ctx);
    if (leg_dim > c.D * c.D) return TN_EINVAL;
    if (!boundary && leg_dim != c.D * c.D) return TN_EINVAL;
    if (leg_dim != c.leg) {               // re-bind the environment with the new leg dimension
        c.leg = leg_dim;
        bind_env(c);
    }
    const size_t n = (size_t)leg_dim * leg_dim * leg_dim * leg_dim;
    for (int t = 0; t < c.nt; ++t)
        TN_CUDA(cudaMemcpyAsync(c.a[0][t], a_host + t * n, n * sizeof(double), cudaMemcpyHostToDevice, c.st));
    if (boundary) {
        TN_CUDA(cudaMemcpyAsync(c.boundary, boundary, leg_dim * sizeof(double), cudaMemcpyHostToDevice, c.st));
    } else {
        std::vector<double> b(c.leg, 0.0);
        for (int i = 0; i < c.D; ++i) b[i * c.D + i] = 1.0;
        TN_CUDA(cudaMemcpyAsync(c.boundary, b.data(), sizeof(double) * c.leg, cudaMemcpyHostToDevice, c.st));
    }
    TN_TRY(ctx_build_network_views(c));
    TN_TRY(ctx_reset_env(c));
    c.have_network = true;
    TN_CUDA(cudaStreamSynchronize(c.st));
    return TN_OK;
}

int tn_reset_env(void* ctx)
{
    if (!ctx) return TN_EINVAL;
    TN_TRY(ctx_reset_env(*C(ctx)));
    TN_CUDA(cudaStreamSynchronize(C(ctx)->st));
    return TN_OK;
}

int tn_ctmrg(void* ctx, double tol, int max_iter, tn_ctm_report* rep)
{
    if (!ctx || max_iter < 1 || !(tol >= 0.0)) return TN_EINVAL;
    Ctx& c = *C(ctx);
    if (!c.have_network) return TN_ESTATE;
    int s = ctmrg_iterations(c, tol, max_iter, rep);
    TN_CUDA(cudaStreamSynchronize(c.st));
    return s;
}

int tn_ctmrg_moves(void* ctx, int n)
{
    if (!ctx || n < 0) return TN_EINVAL;
    Ctx& c = *C(ctx);
    if (!c.have_network) return TN_ESTATE;
    TN_TRY(ctmrg_moves(c, n));
    c.prev_spectra.clear();
    TN_CUDA(cudaStreamSynchronize(c.st));
    return TN_OK;
}

size_t tn_env_size(void* ctx) { return ctx ? C(ctx)->env_size() : 0; }

int tn_get_env(void* ctx, double* host, size_t n)
{
    if (!ctx || !host) return TN_EINVAL;
    Ctx& c = *C(ctx);
    if (n != c.env_size()) return TN_EINVAL;
    TN_CUDA(cudaMemcpyAsync(host, c.envbuf, n * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    TN_CUDA(cudaStreamSynchronize(c.st));
    return TN_OK;
}

int tn_set_env(void* ctx, const double* host, size_t n)
{
    if (!ctx || !host) return TN_EINVAL;
    Ctx& c = *C(ctx);
    if (n != c.env_size()) return TN_EINVAL;
    TN_CUDA(cudaMemcpyAsync(c.envbuf, host, n * sizeof(double), cudaMemcpyHostToDevice, c.st));
    TN_CUDA(cudaStreamSynchronize(c.st));
    c.prev_spectra.clear();
    c.split_ready = true;           // a supplied environment counts as developed
    return TN_OK;
}

int tn_corner_spectra(void* ctx, double* host, size_t n)
{
    if (!ctx || !host) return TN_EINVAL;
    Ctx& c = *C(ctx);
    if (n != (size_t)c.nsites * 4 * c.chi) return TN_EINVAL;
    std::vector<double> s;
    TN_TRY(corner_spectra(c, s));
    std::copy(s.begin(), s.end(), host);
    return TN_OK;
}

int tn_site_scalars(void* ctx, int site, const double* a_host, double out[4])
{
    if (!ctx || !out) return TN_EINVAL;
    Ctx& c = *C(ctx);
    if (site < 0 || site >= c.nsites) return TN_EINVAL;
    const double* da = nullptr;
    size_t mk = c.ar.mark();
    if (a_host) {
        const size_t n = (size_t)c.leg * c.leg * c.leg * c.leg;
        double* t = c.ar.take(n);
        if (!t) return TN_ENOMEM;
        TN_CUDA(cudaMemcpyAsync(t, a_host, n * sizeof(double), cudaMemcpyHostToDevice, c.st));
        da = t;
    }
    int s = site_scalars(c, site, da, out);
    c.ar.release(mk);
    return s;
}

int tn_step_prepare(void* ctx, tn_step_report* rep)
{
    if (!ctx) return TN_EINVAL;
    Ctx& c = *C(ctx);
    if (c.leg != c.D * c.D) { c.leg = c.D * c.D; bind_env(c); TN_TRY(ctx_reset_env(c)); }
    TN_TRY(step_prepare(c, rep));
    TN_CUDA(cudaStreamSynchronize(c.st));
    return TN_OK;
}

int tn_step_update(void* ctx, tn_step_report* rep)
{
    if (!ctx) return TN_EINVAL;
    TN_TRY(step_update(*C(ctx), rep));
    TN_CUDA(cudaStreamSynchronize(C(ctx)->st));
    return TN_OK;
}

int tn_fu_step(void* ctx, double ctm_tol, int ctm_max, tn_step_report* rep)
{
    if (!ctx) return TN_EINVAL;
    tn_step_report r{};
    TN_TRY(tn_step_prepare(ctx, &r));
    tn_ctm_report cr{};
    int s = tn_ctmrg(ctx, ctm_tol, ctm_max, &cr);
    if (s != TN_OK && s != TN_ENOCONV) return s;
    r.ctm_iterations = cr.iterations;
    r.ctm_delta = cr.delta;
    TN_TRY(tn_step_update(ctx, &r));
    if (rep) *rep = r;
    return s;
}

int tn_su_step(void* ctx, tn_step_report* rep)
{
    if (!ctx) return TN_EINVAL;
    tn_step_report r{};
    TN_TRY(su_step(*C(ctx), &r));
    TN_CUDA(cudaStreamSynchronize(C(ctx)->st));
    if (rep) *rep = r;
    return TN_OK;
}

int tn_recycle(void* ctx, int n_re, double* fidelity)
{
    if (!ctx || n_re < 1) return TN_EINVAL;
    TN_TRY(recycle(*C(ctx), n_re, fidelity));
    TN_CUDA(cudaStreamSynchronize(C(ctx)->st));
    return TN_OK;
}

// Recycling windows can go unstable when the recycled environment no longer
// fits the state (Sec. VI.D and Sec. VII): a window is judged unstable when the
// gauge-fix fidelity F of Eq. (25) falls below opts->min_fidelity, or when a
// recycled step produces a non-finite tensor.  Such a window is redone as plain
// full-update steps, starting from the plain step the window's environment
// computation already produced (its result is kept in Asave), and the window
// length is halved for the rest of the evolution (at least 1).
static int save_state(Ctx& c)
{
    const size_t per = 2 * (size_t)c.D * c.D * c.D * c.D;
    for (int t = 0; t < c.nt; ++t)
        TN_CUDA(cudaMemcpyAsync(c.Asave[t], c.A[t], per * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
    return TN_OK;
}

static int restore_state(Ctx& c)
{
    const size_t per = 2 * (size_t)c.D * c.D * c.D * c.D;
    for (int t = 0; t < c.nt; ++t)
        TN_CUDA(cudaMemcpyAsync(c.A[t], c.Asave[t], per * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
    c.have_gate = false;
    return TN_OK;
}

static bool window_unstable(double F, const tn_evolve_opts* o)
{
    return !std::isfinite(F) || (o->min_fidelity > 0.0 && F < o->min_fidelity);
}

// One plain full-update step inside tn_evolve (an environment computation).
static int plain_step(void* ctx, const tn_evolve_opts* o, tn_evolve_report& r)
{
    tn_step_report sr{};
    int s = tn_fu_step(ctx, o->ctm_tol, o->ctm_max, &sr);
    if (s == TN_ENOCONV) r.nonconverged++;
    else if (s != TN_OK) return s;
    r.env_computations++;
    r.ctm_iterations += sr.ctm_iterations;
    return TN_OK;
}

// Recycling with the threshold trigger: a window starts with an environment
// computation (a plain step; its bond environments N_0 are kept) and continues
// with recycled steps from A_0; after every check_every steps one warm CTMRG
// iteration on the current state gives its bond environments N (a8), and the
// window ends once max_links ||N - N_0||_F / ||N_0||_F > eps, or after n_re steps.
static int evolve_threshold(Ctx& c, void* ctx, int n_steps, const tn_evolve_opts* o, tn_evolve_report& r,
                            int& n_re)
{
    const int k = c.kD;
    const size_t n4 = (size_t)k * k * k * k;
    int done = 0;
    while (done < n_steps) {
        TN_TRY(plain_step(ctx, o, r));
        TN_CUDA(cudaMemcpyAsync(c.N4ref, c.N4[0], sizeof(double) * n4 * c.nl, cudaMemcpyDeviceToDevice, c.st));
        TN_TRY(save_state(c));                       // the plain step's result
        double F = 0.0;
        TN_TRY(recycle_build(c, &F));
        r.last_fidelity = F;
        if (window_unstable(F, o)) {                 // keep the plain step, shorten later windows
            TN_TRY(restore_state(c));
            ++done;
            r.fallbacks++;
            n_re = std::max(1, n_re / 2);
            continue;
        }
        const int start = done;
        for (int w = 1; done < n_steps && w <= n_re; ++w) {
            int s = recycle_advance(c, 1);
            if (s == TN_ENUMERIC) {                  // undo the window: back to its plain step
                TN_TRY(restore_state(c));
                done = start + 1;
                r.fallbacks++;
                n_re = std::max(1, n_re / 2);
                break;
            }
            TN_TRY(s);
            ++done;
            if (w % o->check_every != 0 || done >= n_steps) continue;
            TN_TRY(step_prepare(c, nullptr));
            tn_ctm_report cr{};
            int cs = ctmrg_iterations(c, 0.0, 1, &cr);
            if (cs != TN_OK && cs != TN_ENOCONV) return cs;
            r.ctm_iterations += 1;
            TN_TRY(bond_envs_psd(c));
            c.prepared = false;
            double d = 0.0;
            TN_TRY(env_change(c, &d));
            r.checks++;
            r.last_change = d;
            if (!(d <= o->recycle_eps)) break;
        }
    }
    r.steps = done;
    return TN_OK;
}

int tn_evolve(void* ctx, int n_steps, const tn_evolve_opts* o, tn_evolve_report* rep)
{
    if (!ctx || !o || n_steps < 0) return TN_EINVAL;
    if (o->recycle < TN_RECYCLE_OFF || o->recycle > TN_RECYCLE_THRESHOLD) return TN_EINVAL;
    if (o->recycle != TN_RECYCLE_OFF && o->n_re < 1) return TN_EINVAL;
    if (o->recycle == TN_RECYCLE_THRESHOLD && (o->check_every < 1 || o->recycle_eps != o->recycle_eps))
        return TN_EINVAL;
    if (o->warmup_plain < 0 || o->min_fidelity != o->min_fidelity) return TN_EINVAL;
    Ctx& c = *C(ctx);
    c.als_tol = o->als_tol > 0.0 ? o->als_tol : 1e-12;
    c.als_max = o->als_max > 0 ? o->als_max : 50;
    tn_evolve_report r{};
    long long moves0 = c.ctm_moves;
    int done = 0;
    int n_re = o->n_re;
    // warm-up: plain steps first (the recycled windows start from an evolved state)
    const int warm = o->recycle == TN_RECYCLE_OFF ? 0 : std::min(o->warmup_plain, n_steps);
    for (; done < warm; ++done) TN_TRY(plain_step(ctx, o, r));
    if (o->recycle == TN_RECYCLE_THRESHOLD) {
        TN_TRY(evolve_threshold(c, ctx, n_steps - done, o, r, n_re));
        r.steps += done;
    } else {
        while (done < n_steps) {
            TN_TRY(plain_step(ctx, o, r));
            if (!o->recycle) { done += 1; continue; }
            const int k = std::min(n_re, n_steps - done);
            TN_TRY(save_state(c));                   // the plain step's result
            double F = 0.0;
            TN_TRY(recycle_build(c, &F));
            r.last_fidelity = F;
            int s = window_unstable(F, o) ? TN_EUNSTABLE : recycle_advance(c, k);
            if (s == TN_EUNSTABLE || s == TN_ENUMERIC) {
                // redo the window as plain steps: its first step is the one just computed
                TN_TRY(restore_state(c));
                for (int j = 1; j < k; ++j) TN_TRY(plain_step(ctx, o, r));
                r.fallbacks++;
                n_re = std::max(1, n_re / 2);
            } else {
                TN_TRY(s);
            }
            done += k;
        }
        r.steps = done;
    }
    r.ctm_moves = (int)(c.ctm_moves - moves0);
    r.final_n_re = n_re;
    TN_CUDA(cudaStreamSynchronize(c.st));
    if (rep) *rep = r;
    return r.fallbacks ? TN_EUNSTABLE : TN_OK;
}

// Batched form: independent contexts evolved concurrently, one host thread per
// context at a time, each context on its own stream (so their kernels overlap).
int tn_evolve_batch(void** ctxs, int n_ctx, int n_steps, const tn_evolve_opts* opts, int n_threads, int* statuses,
                    tn_evolve_report* reps)
{
    if (!ctxs || n_ctx < 1 || !opts || n_steps < 0) return TN_EINVAL;
    for (int i = 0; i < n_ctx; ++i) {
        if (!ctxs[i]) return TN_EINVAL;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i] || (C(ctxs[j])->st == C(ctxs[i])->st)) return TN_EINVAL;   // shared stream
    }
    int dev = 0;
    TN_CUDA(cudaGetDevice(&dev));
    const int nt = std::max(1, std::min(n_threads > 0 ? n_threads : n_ctx, n_ctx));
    std::atomic<int> next{0};
    std::vector<int> st(n_ctx, TN_OK);
    std::vector<tn_evolve_report> rp(n_ctx);
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (int i = next.fetch_add(1); i < n_ctx; i = next.fetch_add(1))
            st[i] = tn_evolve(ctxs[i], n_steps, opts, &rp[i]);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
    int first = TN_OK;
    for (int i = 0; i < n_ctx; ++i) {
        if (statuses) statuses[i] = st[i];
        if (reps) reps[i] = rp[i];
        if (first == TN_OK && st[i] != TN_OK && st[i] != TN_EUNSTABLE) first = st[i];
    }
    return first;
}

int tn_set_autotune(int enable)
{
    set_autotune(enable);
    return autotune_entries();
}

int tn_measure(void* ctx, tn_observables* obs)
{
    if (!ctx || !obs) return TN_EINVAL;
    Ctx& c = *C(ctx);
    if (!c.have_state) return TN_ESTATE;
    return measure(c, obs);
}

int tn_get_tensor(void* ctx, int which, int index, double* host, size_t n)
{
    if (!ctx || !host) return TN_EINVAL;
    Ctx& c = *C(ctx);
    const int D = c.D, k = c.kD;
    const double* src = nullptr;
    size_t size = 0;
    auto tid_ok = [&]() { return index >= 0 && index < c.nt; };
    auto link_ok = [&]() { return index >= 0 && index < c.nl; };
    switch (which) {
        case TN_T_STATE: if (!tid_ok()) return TN_EINVAL; src = c.A[index]; size = 2 * (size_t)D * D * D * D; break;
        case TN_T_CANON: if (!tid_ok()) return TN_EINVAL; src = c.Ac[index]; size = 2 * (size_t)D * D * D * D; break;
        case TN_T_LAMBDA: if (!link_ok()) return TN_EINVAL; src = c.lam[index]; size = D; break;
        case TN_T_THETA: if (!tid_ok()) return TN_EINVAL; src = c.Theta[index]; size = 2 * (size_t)k * k * k * k; break;
        case TN_T_PRE_P: if (!link_ok()) return TN_EINVAL; src = c.preP[index]; size = (size_t)k * D; break;
        case TN_T_PRE_Q: if (!link_ok()) return TN_EINVAL; src = c.preQ[index]; size = (size_t)k * D; break;
        case TN_T_DOUBLE: if (!tid_ok()) return TN_EINVAL; src = c.a[0][index]; size = (size_t)c.leg * c.leg * c.leg * c.leg; break;
        case TN_T_BOND_ENV: if (!link_ok()) return TN_EINVAL; src = c.N4[index]; size = (size_t)k * k * k * k; break;
        case TN_T_FU_P: if (!link_ok()) return TN_EINVAL; src = c.fuP[index]; size = (size_t)k * D; break;
        case TN_T_FU_Q: if (!link_ok()) return TN_EINVAL; src = c.fuQ[index]; size = (size_t)k * D; break;
        case TN_T_GAUGE_W: if (!link_ok()) return TN_EINVAL; src = c.W[index]; size = (size_t)D * D; break;
        case TN_T_GATE_K: if (index < 0 || index >= 4 * c.nt) return TN_EINVAL; src = c.K[index / 4][index % 4]; size = (size_t)k * D; break;
        case TN_T_PEPO: src = c.g; size = 64; break;
        default: return TN_EINVAL;
    }
    if (n != size) return TN_EINVAL;
    TN_CUDA(cudaMemcpyAsync(host, src, size * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    TN_CUDA(cudaStreamSynchronize(c.st));
    return TN_OK;
}

int tn_gemm_f64(int transA, int transB, int m, int n, int k, double alpha,
                const double* dA, int lda, long long strideA,
                const double* dB, int ldb, long long strideB, double beta,
                double* dC, int ldc, long long strideC, int batch, void* stream)
{
    if (m < 0 || n < 0 || k < 0 || batch < 0 || (m * n > 0 && (!dA || !dB || !dC))) return TN_EINVAL;
    return gemm(reinterpret_cast<cudaStream_t>(stream), transA != 0, transB != 0, m, n, k, alpha,
                dA, lda, strideA, dB, ldb, strideB, beta, dC, ldc, strideC, batch);
}

int tn_set_projector_cutoff(void* ctx, double cut)
{
    if (!ctx || cut != cut) return TN_EINVAL;
    static_cast<Ctx*>(ctx)->cut_override = cut < 0.0 ? -1.0 : cut;
    return TN_OK;
}

// tensor-core kind of a split precision form (-1: not a split form)
static int split_kind(int precision)
{
    switch (precision) {
        case TN_TF32X3: return 0;
        case TN_BF16X3: return 1;
        case TN_BF16S4: return 2;
        case TN_F64S7: return 3;
        default: return -1;
    }
}

size_t tn_gemm_split_workspace_bytes(int precision, int m, int n, int k)
{
    if (split_kind(precision) < 0 || m < 1 || n < 1 || k < 1) return 0;
    return gemm_tc_scratch_bytes(split_kind(precision), m, n, k);
}

int tn_gemm_split(int precision, int transA, int transB, int m, int n, int k, double alpha,
                  const double* dA, int lda, const double* dB, int ldb, double beta,
                  double* dC, int ldc, void* d_workspace, size_t workspace_bytes, void* stream)
{
    if (split_kind(precision) < 0) return TN_EINVAL;
    if (m < 1 || n < 1 || k < 1 || !dA || !dB || !dC || !d_workspace) return TN_EINVAL;
    if (lda < (transA ? m : k) || ldb < (transB ? k : n) || ldc < n) return TN_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256) return TN_EINVAL;
    const int kind = split_kind(precision);
    if (workspace_bytes < gemm_tc_scratch_bytes(kind, m, n, k)) return TN_ENOMEM;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Arena ar;
    ar.base = static_cast<char*>(d_workspace);
    ar.cap = workspace_bytes;
    TN_TRY(gemm_tc(st, ar, kind, transA != 0, transB != 0, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc));
    int flag = 0;
    TN_TRY(tc_status(st, &flag));
    return flag ? TN_ETIMEOUT : TN_OK;
}

int tn_fp64_rate_probe(int iters, double* flops, void* stream)
{
    if (iters < 1 || !flops) return TN_EINVAL;
    return dfma_probe(reinterpret_cast<cudaStream_t>(stream), iters, flops);
}

int tn_selftest_wait_timeout(void* stream)
{
    int flag = 0;
    TN_TRY(wait_selftest(reinterpret_cast<cudaStream_t>(stream), &flag));
    return flag ? TN_ETIMEOUT : TN_OK;
}

int tn_permute_f64(const double* d_in, double* d_out, int rank, const int* dims, const int* perm, void* stream)
{
    if (!d_in || !d_out || !dims || !perm || rank < 1 || rank > 8) return TN_EINVAL;
    for (int i = 0; i < rank; ++i) if (dims[i] < 0) return TN_EINVAL;
    bool seen[8] = {false};
    for (int i = 0; i < rank; ++i) { if (perm[i] < 0 || perm[i] >= rank || seen[perm[i]]) return TN_EINVAL; seen[perm[i]] = true; }
    return permute(reinterpret_cast<cudaStream_t>(stream), d_in, d_out, rank, dims, perm);
}

int tn_svd_small(const double* dA, int m, int n, int batch, double* dU, double* dS, double* dV, void* stream)
{
    if (!dA || !dU || !dS || !dV) return TN_EINVAL;
    return svd_small(reinterpret_cast<cudaStream_t>(stream), dA, m, n, batch, dU, dS, dV);
}

int tn_eigh_small(const double* dA, int n, int batch, double* dW, double* dV, void* stream)
{
    if (!dA || !dW || !dV) return TN_EINVAL;
    return eigh_small(reinterpret_cast<cudaStream_t>(stream), dA, n, batch, dW, dV);
}

int tn_truncated_svd(void* ctx, const double* dM, int m, int k, double* dU, double* dS, double* dV, const double* warm)
{
    if (!ctx || !dM || !dU || !dS || !dV || m < 1 || k < 1 || k > m || k > 96) return TN_EINVAL;
    Ctx& c = *C(ctx);
    TsvdStats st;
    int s = truncated_svd(c.st, c.ar, dM, m, k, dU, dS, dV, warm, &st);
    TN_CUDA(cudaStreamSynchronize(c.st));
    return s;
}

}  // extern "C"
