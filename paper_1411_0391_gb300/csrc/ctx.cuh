// Context of the tnite library: configuration, device buffers (all carved from
// the caller's workspace) and the frame bookkeeping of the CTMRG.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace tn {

constexpr int MAXT = 2;        // tensor ids per cell
constexpr int MAXL = 4;        // link types per cell
constexpr int MAXS = 4;        // sites per cell

// Environment of one site: C1..C4 then T1..T4 (clockwise in/out legs).
struct Env { double* C[4]; double* T[4]; };

// A view of the network after r counter-clockwise rotations: cell geometry,
// which stored environment plays which role, and which rotated double layer
// sits on each tensor id.  Rotations only relabel pointers.
struct Frame {
    int Lx, Ly, rot;
    int pat[4][4];             // pat[y][x] = tensor id
    Env env[MAXS];             // env[y*Lx + x]
    int tid(int x, int y) const { x %= Lx; if (x < 0) x += Lx; y %= Ly; if (y < 0) y += Ly; return pat[y][x]; }
    Env& e(int x, int y) { x %= Lx; if (x < 0) x += Lx; y %= Ly; if (y < 0) y += Ly; return env[y * Lx + x]; }
    Frame rotated() const;
};

struct Ctx {
    tn_config cfg;
    cudaStream_t st = nullptr;
    Arena ar;
    size_t scratch_base = 0;

    int nt = 0, nl = 0, Lx = 0, Ly = 0, nsites = 0;
    int pat[4][4];
    int D = 0, chi = 0, kD = 0, leg = 0;   // leg: dimension of a double-layer leg
    double J = 1.0, h = 0.0, tau = 0.0;
    double als_tol = 1e-12;    // ALS stop: ||M_new - M|| <= als_tol ||M|| (reading of Sec. VI.B)
    int als_max = 50;
    bool have_state = false, have_network = false, have_pepo = false, prepared = false, updated = false;
    bool have_gate = false;    // the leg matrices K of a recycling window are built

    // state and step tensors
    double* A[MAXT];
    double* Ac[MAXT];          // weighted canonical form (a11)
    double* A0[MAXT];          // recycling reference
    double* A1[MAXT];          // pre-truncated sites / canonical form of the updated state
    double* Asave[MAXT];       // the plain-step result of a recycling window (fallback)
    double* lam[MAXL];
    double* cmaps[MAXT][4];    // canonical leg maps of the last canonicalisation (D x D)
    double* g = nullptr;       // iPEPO d*d*16
    double* Theta[MAXT];
    double* preP[MAXL];
    double* preQ[MAXL];
    double* N4[MAXL];
    double* N4ref = nullptr;   // bond environments at the start of a recycling window (all links)
    double* fuP[MAXL];
    double* fuQ[MAXL];
    double* W[MAXL];
    double* K[MAXT][4];
    // network and environment
    double* a[4][MAXT];        // double layer per rotation and tensor id, leg^4
    double* ab[4][MAXT][4];    // a transposed for enlarged corner type c (UL, UR, LR, LL)
    double* aT4[4][MAXT];      // a[l][d][r][u] for the edge renormalisation
    double* boundary = nullptr;
    double* envbuf = nullptr;
    Env env0[MAXS];            // environment storage in the unrotated frame
    double* warmV[4][4][4];    // projector right vectors (rotation, x, y) for warm starts
    bool warm_ok[4][4][4];
    double cut_override = -1.0;   // projector cutoff set by tn_set_projector_cutoff (< 0: default)
    // Precision schedule of the split forms: after an environment reset the
    // moves run in FP64 until the environment has developed (corner spectra
    // within 1e-4 of the previous iteration, or 32 moves); only then the
    // contractions switch to the tensor cores.  From the low-rank start the
    // loop matrix has many directions at the product-error level, which
    // S^{-1/2} amplifies into a wrong fixed point.
    bool split_ready = false;
    int fp64_moves = 0;
    double* Pup[4];            // projectors of the current column, per y
    double* Plo[4];
    double* dscratch = nullptr;   // small device scratch (reports)
    // streams and events of the concurrent cuts of a column (created with the context)
    cudaStream_t cut_st[MAXS] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[MAXS] = {nullptr, nullptr, nullptr, nullptr};
    ~Ctx()
    {
        for (int i = 0; i < MAXS; ++i) {
            if (cut_st[i]) cudaStreamDestroy(cut_st[i]);
            if (ev_join[i]) cudaEventDestroy(ev_join[i]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
    }
    double* hbuf = nullptr;

    long long ctm_moves = 0;
    long long svd_calls = 0, svd_iterations = 0;
    std::vector<double> prev_spectra;

    int N() const { return chi * leg; }
    // contraction arithmetic of the CTMRG moves now: -1 FP64, 0 TF32 x3, 1 BF16 x3,
    // 2 BF16 integer slices (4) with exact accumulation, 3 the same with 7 slices
    int kind() const
    {
        if (cfg.precision == TN_F64S7) return 3;      // FP64-accurate: no FP64 start needed
        if (!split_ready) return -1;
        switch (cfg.precision) {
            case TN_TF32X3: return 0;
            case TN_BF16X3: return 1;
            case TN_BF16S4: return 2;
            default: return -1;
        }
    }
    // arithmetic of the products with the loop matrix inside the projector SVD:
    // FP64 SIMT, or 7-slice FP64-accurate tensor-core products for the slice forms
    int svd_kind() const
    {
        return (cfg.precision == TN_BF16S4 || cfg.precision == TN_F64S7) ? 3 : -1;
    }
    // Ritz residual threshold (relative to s_1) of the FP64 projector SVD: the loop
    // matrix of the precision form is itself known only to the accuracy of its
    // split products (~1e-7 TF32 x3, ~4e-6 BF16 x3, ~1e-9 BF16 slices), so
    // resolving it further than 1e-10 (1e-9, 1e-12) buys nothing
    double svd_tol() const
    {
        switch (kind()) {
            case 0: return 1e-10;
            case 1: return 1e-9;
            case 2: return 1e-12;
            default: return 1e-13;
        }
    }
    // inverse-square-root cutoff of the projectors (relative to s_1): singular
    // values of the loop matrix below it are dropped (1e-12 unless overridden)
    double proj_cut() const { return cut_override >= 0.0 ? cut_override : 1e-12; }
    size_t env_size() const { return (size_t)nsites * (4 * (size_t)chi * chi + 4 * (size_t)chi * chi * leg); }
    Frame frame0();
};

// ctmrg.cu
int ctx_build_network_views(Ctx& c);                  // a -> rotations, ab, aT4
int ctx_reset_env(Ctx& c);
int ctmrg_move(Ctx& c, Frame& f);                      // one left move in frame f
int ctmrg_iterations(Ctx& c, double tol, int max_iter, tn_ctm_report* rep);
int ctmrg_moves(Ctx& c, int n);
int corner_spectra(Ctx& c, std::vector<double>& out);
int site_scalars(Ctx& c, int site, const double* d_a, double out[4]);

// step.cu
int build_pepo(Ctx& c);
int build_double_layers(Ctx& c, double* const* sites, int Dsite);
int canonicalize(Ctx& c, double* const* A, double* const* Aout, int* iters, bool keep_maps);
int step_prepare(Ctx& c, tn_step_report* rep);
int step_update(Ctx& c, tn_step_report* rep);
int su_step(Ctx& c, tn_step_report* rep);
int recycle(Ctx& c, int n_re, double* F);
int recycle_build(Ctx& c, double* F);
int recycle_advance(Ctx& c, int n_re);
int bond_envs_psd(Ctx& c);
int env_change(Ctx& c, double* out);
int measure(Ctx& c, tn_observables* obs);
int state_finite(Ctx& c, double* const* T, bool* ok);   // ok = no NaN/Inf in the cell's tensors

}  // namespace tn
