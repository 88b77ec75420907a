/*
 * tnite.h - C ABI of the GB300 (sm_103a) library for imaginary-time evolution
 * of an infinite PEPS with CTMRG environments, full-update truncation and
 * environment recycling.
 *
 * Method: Phien, McCulloch, Vidal, "Faster convergence of imaginary time
 * evolution tensor network algorithms by recycling the environment"
 * (arXiv:1411.0391).  Section/equation numbers below refer to that paper.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All floating point data is IEEE double, row-major (C order).
 *  - Site tensor A[s][l][r][d][u], physical dimension d = 2, bond dimension D;
 *    x grows to the right, y downward; A's r leg joins the l leg of the site
 *    to its right, its d leg the u leg of the site below.
 *  - Unit cells: TN_CELL_CHECKERBOARD holds tensors A (id 0) and B (id 1) in
 *    the pattern [[A, B], [B, A]]; TN_CELL_SINGLE holds one tensor.
 *  - A "state" buffer is the concatenation of the cell's tensors in id order,
 *    n_tensors * d * D^4 doubles.
 *  - Status codes: every int-returning call returns TN_OK (0) or a negative
 *    TN_E* code; tn_strerror() gives a message.  TN_ENOCONV is a warning: the
 *    results are written and usable, an iteration cap was hit.
 *  - Ownership: the caller owns every host and device buffer it passes.  A
 *    context never allocates device memory: all of it is carved from the
 *    device workspace given to tn_create (size from tn_workspace_bytes).
 *    Host buffers may be freed as soon as a call returns (the library copies).
 *  - Streams: a context enqueues all its work on the CUDA stream given to
 *    tn_create and synchronises that stream before returning from any call
 *    that reports host-visible results.  A context is not thread-safe.
 */
#ifndef TNITE_H
#define TNITE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define TN_OK         0
#define TN_EINVAL    -1   /* bad argument: null pointer, size, D > chi, tau <= 0 ... */
#define TN_ENOMEM    -2   /* workspace too small */
#define TN_ECUDA     -3   /* a CUDA runtime call failed */
#define TN_ENOCONV   -4   /* iteration cap reached (warning; results written) */
#define TN_ENUMERIC  -5   /* NaN or Inf detected */
#define TN_ESTATE    -6   /* call out of order (e.g. no state set) */
#define TN_ESCRATCH  -7   /* problem larger than the fixed scratch of tn_truncated_svd_noalloc */
#define TN_ETIMEOUT  -8   /* a bounded device-side wait expired (tensor-core kernels); results invalid */
#define TN_EUNSTABLE -9   /* warning from tn_evolve: some recycling windows were judged unstable and
                             redone as plain steps (results written and usable) */

/* ---- configuration ------------------------------------------------------ */
#define TN_CELL_CHECKERBOARD 2
#define TN_CELL_SINGLE       1

#define TN_F64    0   /* every contraction in double */
#define TN_TF32X3 1   /* split-precision tensor-core products, TF32 head + tail (tn_gemm_split) */
#define TN_BF16X3 2   /* split-precision tensor-core products, BF16 head + tail (tn_gemm_split) */
#define TN_BF16S4 3   /* exact-accumulation tensor-core products: 4 BF16 integer slices per operand
                         (the Ozaki scheme), 10 slice products, FP32 accumulation that is exact
                         by construction; error per term of the K sum below 5 * 2^-32 of the
                         row/column scales (tn_gemm_split) */
#define TN_F64S7  4   /* FP64-accurate tensor-core products: 7 BF16 integer slices per operand,
                         28 slice products, exact accumulation; error per term below
                         8 * 2^-56 = 2^-53 of the row/column scales, the unit roundoff of
                         FP64 (tn_gemm_split) */

typedef struct tn_config {
    int D;          /* PEPS bond dimension, 1..8 */
    int chi;        /* CTM bond dimension, 1 <= chi <= 96 */
    int cell;       /* TN_CELL_CHECKERBOARD or TN_CELL_SINGLE */
    int precision;  /* arithmetic of the CTMRG contractions (C.T, enlarged
                       corners, half-system and loop products, projector
                       products, renormalisation): TN_F64, TN_TF32X3,
                       TN_BF16X3, TN_BF16S4 or TN_F64S7.  With TN_BF16S4
                       and TN_F64S7 the products with the loop matrix inside
                       the projector SVD run as 7-slice (FP64-accurate)
                       tensor-core products too; TN_F64S7 needs no FP64 start.  The split forms start in FP64 after
                       tn_reset_env and switch once the environment has
                       developed (corner spectra within 1e-4 between
                       iterations, or 32 moves); an environment given by
                       tn_set_env counts as developed.  The projector SVD,
                       bond environment, full-update solve, gauge fixing and
                       observables are FP64 in every mode. */
} tn_config;

/* Number of kernels this library has launched in the process so far (all
 * contexts); a monotone counter for accounting, no synchronisation implied. */
unsigned long long tn_launch_count(void);

/* Bytes of device workspace a context with this configuration needs
 * (256-byte aligned base).  Returns 0 for an invalid configuration. */
size_t tn_workspace_bytes(const tn_config* cfg);

/* Create a context.  d_workspace: device pointer of at least
 * tn_workspace_bytes(cfg) bytes, owned by the caller and kept alive until
 * tn_destroy.  stream: a cudaStream_t (NULL = legacy default stream). */
int  tn_create(void** out_ctx, const tn_config* cfg, void* d_workspace,
               size_t workspace_bytes, void* stream);
void tn_destroy(void* ctx);
const char* tn_strerror(int status);

/* ---- problem definition (Sec. V.A, VI.A) -------------------------------- */
/* Transverse-field Ising model H = -J sum_<ij> Z_i Z_j - h sum_i X_i.
 * Reading: J = 1 is the paper's model; other J > 0 rescale the ZZ term. */
int tn_set_hamiltonian(void* ctx, double J, double h);
/* Trotter step tau > 0: rebuilds the iPEPO g of Sec. VI.A, Fig. 20 (row a1):
 * g = g_F (bond halves on l, r, d, u) g_F, kappa = 2. */
int tn_set_time_step(void* ctx, double tau);

/* Copy the iPEPS tensors in (n = n_tensors*d*D^4 doubles, host memory). */
int tn_set_state(void* ctx, const double* host, size_t n);
int tn_get_state(void* ctx, double* host, size_t n);

/* ---- environment: CTMRG (Sec. VI.B item 1, Fig. 21a; rows a2-a6) -------- */
typedef struct tn_ctm_report {
    int    iterations;   /* CTMRG iterations done (one = left, up, right, down move) */
    int    converged;    /* 1 if delta < tol */
    double delta;        /* max over corners of ||s_new - s_old||_2 of the
                            sum-normalised corner singular values */
    int    svd_calls;    /* projector SVDs computed in this call */
    int    svd_iterations; /* subspace iterations summed over those SVDs */
} tn_ctm_report;

/* Build the double layers a = sum_s A^s (x) A^s of the current state (row a2),
 * with the ket and bra legs fused ket*D + bra. */
int tn_build_double_layer(void* ctx);
/* Replace the double layers by an arbitrary network: a_host holds one tensor
 * a[l][r][d][u] per tensor id, each leg of dimension leg_dim (leg_dim <= D^2
 * of the configuration); boundary (leg_dim doubles) is the vector of the
 * trivial initial boundary (NULL: the ket-bra identity, leg_dim = D^2). */
int tn_set_network(void* ctx, const double* a_host, int leg_dim, const double* boundary);
/* Reset the environment to the trivial boundary (bond 1 padded to chi). */
int tn_reset_env(void* ctx);
/* Run CTMRG iterations on the current double layers, warm-started from the
 * context's environment, until the corner-spectrum change is below tol or
 * max_iter iterations.  Returns TN_OK or TN_ENOCONV. */
int tn_ctmrg(void* ctx, double tol, int max_iter, tn_ctm_report* rep);
/* Run n_moves directional moves (left, up, right, down, left, ...) without a
 * convergence test; a move absorbs every column of the cell (rows a3-a5). */
int tn_ctmrg_moves(void* ctx, int n_moves);
/* Environment in/out: per site (x, y) in row-major cell order, C1..C4
 * (chi x chi each) then T1..T4 (chi x chi x leg_dim each), C[in][out] and
 * T[in][out][m] with the clockwise in/out convention of Fig. 21a. */
size_t tn_env_size(void* ctx);
int tn_get_env(void* ctx, double* host, size_t n);
int tn_set_env(void* ctx, const double* host, size_t n);
/* Corner spectra (row a6): s / sum(s) of every corner, sorted descending:
 * out[(site*4 + corner)*chi + i]; n = n_sites*4*chi. */
int tn_corner_spectra(void* ctx, double* host, size_t n);
/* Contractions of one site's environment with a tensor a (leg_dim legs):
 * out[0] = Z1 (with a), out[1] = Z0 (corners only), out[2] = Zh (T1, T3),
 * out[3] = Zv (T2, T4); a_host NULL uses the site's own double layer. */
int tn_site_scalars(void* ctx, int site, const double* a_host, double out[4]);

/* ---- one imaginary-time step (Sec. VI.B, VI.C; rows a1, a7-a13) --------- */
typedef struct tn_step_report {
    int    canon_iters;     /* canonical-form iterations of the state (a11) */
    int    ctm_iterations;  /* CTMRG iterations of this step (a3-a6) */
    double ctm_delta;
    int    als_iters[8];    /* ALS sweeps per link type (a9) */
    double als_cost[8];     /* final cost f / <g|g> per link type */
} tn_step_report;

/* Prepare a full-update step: canonical form of the state (a11, with its
 * weights lambda), Theta = g A_c (a1), simple-update pre-truncation (a7) and
 * the double layers of the pre-truncated tensors (a2). */
int tn_step_prepare(void* ctx, tn_step_report* rep);
/* Bond environment (a8), ALS (a9) and assembly (a10) on every link type; the
 * state becomes A~ = Q Theta P (max-abs normalised).  Requires a prior
 * tn_step_prepare and tn_ctmrg. */
int tn_step_update(void* ctx, tn_step_report* rep);
/* Plain full-update step: prepare, CTMRG(ctm_tol, ctm_max), update.
 * tn_step_prepare, tn_step_update, tn_fu_step, tn_su_step and tn_recycle
 * return TN_ENUMERIC when the state they start from or produce holds a NaN
 * or Inf (the check runs on the device before and after the step). */
int tn_fu_step(void* ctx, double ctm_tol, int ctm_max, tn_step_report* rep);

/* One simple-update step (no environment): canonical form, Theta = gA, and
 * every leg truncated kappa*D -> D by the lambda-weighted simple-update
 * projectors (Sec. VI.B, last paragraph; the method Sec. VI.D compares the
 * full update with).  The state is replaced and max-abs normalised; the
 * environment is left as it was.  rep (optional): canon_iters. */
int tn_su_step(void* ctx, tn_step_report* rep);

/* Recycling window of Sec. VI.C: after tn_step_prepare + tn_ctmrg +
 * tn_step_update, build the renormalised gate (canonical form of A~ (a11),
 * gauge fix against A_0 (a12), leg matrices K (a13)); the state is reset to
 * A_0 and then advanced by n_re applications A <- (g A) x_legs K.
 * fidelity (optional out): the local fidelity F of Eq. (25). */
int tn_recycle(void* ctx, int n_re, double* fidelity);

#define TN_RECYCLE_OFF        0   /* plain full update every step */
#define TN_RECYCLE_FIXED      1   /* windows of n_re steps per environment (Sec. VI.C) */
#define TN_RECYCLE_THRESHOLD  2   /* windows that end when the bond environment drifts */

typedef struct tn_evolve_opts {
    int    recycle;        /* TN_RECYCLE_OFF / _FIXED / _THRESHOLD */
    int    n_re;           /* FIXED: steps per environment computation;
                              THRESHOLD: the longest window */
    double ctm_tol;        /* CTMRG tolerance per environment computation */
    int    ctm_max;        /* CTMRG iteration cap */
    double recycle_eps;    /* THRESHOLD: end the window once max over link types of
                              ||N - N_0||_F / ||N_0||_F exceeds it (N_0: the bond
                              environments of the window's environment computation,
                              N: those of the current state after one warm CTMRG
                              iteration, both normalised and positive as in a8) */
    int    check_every;    /* THRESHOLD: recycled steps between checks (>= 1) */
    int    warmup_plain;   /* plain full-update steps before the first recycling
                              window (counted in n_steps) */
    double als_tol;        /* ALS stop (relative change of PQ); <= 0: 1e-12 */
    int    als_max;        /* ALS sweep cap; <= 0: 50 */
    double min_fidelity;   /* instability test of a recycling window (Sec. VI.D, VII): a window
                              whose gauge-fix fidelity F (Eq. 25) is below it, or whose recycled
                              steps produce a NaN/Inf, is redone as plain full-update steps and
                              the window length is halved from then on (at least 1); <= 0
                              disables the F test (the NaN/Inf test always applies) */
} tn_evolve_opts;

typedef struct tn_evolve_report {
    int    steps;          /* imaginary-time steps done */
    int    env_computations;
    int    ctm_iterations; /* total CTMRG iterations (checks included) */
    int    ctm_moves;      /* total directional moves */
    int    nonconverged;   /* environment computations that hit ctm_max */
    double last_fidelity;  /* F of the last recycling window */
    int    checks;         /* THRESHOLD: bond-environment checks made */
    double last_change;    /* THRESHOLD: the last measured change */
    int    fallbacks;      /* recycling windows judged unstable and redone as plain steps */
    int    final_n_re;     /* the window length in force at the end */
} tn_evolve_report;

/* n_steps imaginary-time steps (Sec. VI.B-C).  The threshold mode is the
 * reading of "the environment recycled until the bond-environment change
 * exceeds eps" (the paper itself uses a fixed N_Re).  The ALS settings stay
 * in force for later tn_fu_step / tn_step_update calls.  TN_EINVAL for an
 * unknown mode, n_re < 1 when recycling, check_every < 1, a NaN eps or
 * min_fidelity, or a negative warmup_plain.  Returns TN_OK, TN_EUNSTABLE
 * (warning: rep->fallbacks windows were redone without recycling) or an
 * error; TN_ENUMERIC when a plain step produces a NaN/Inf. */
int tn_evolve(void* ctx, int n_steps, const tn_evolve_opts* opts, tn_evolve_report* rep);

/* Batched form (no counterpart in the paper: many independent instances, e.g.
 * several fields h, bond dimensions D and chi, at once).  ctxs: n_ctx contexts
 * created by the caller, each with its own CUDA stream (TN_EINVAL if two share
 * a context or a stream); every one is evolved n_steps with the same options
 * by a pool of min(n_threads, n_ctx) host threads (n_threads <= 0: one per
 * context), so the kernels of different instances run concurrently on the
 * GPU.  statuses[i], reps[i] (optional, n_ctx entries) receive each tn_evolve
 * result.  Every context must live on the device that is current in the
 * calling thread (the worker threads make that device current).  Returns
 * TN_OK when every instance returned TN_OK or TN_EUNSTABLE, else the first
 * other status.  No other thread may use the contexts while the call runs. */
int tn_evolve_batch(void** ctxs, int n_ctx, int n_steps, const tn_evolve_opts* opts, int n_threads,
                    int* statuses, tn_evolve_report* reps);

/* Tile autotuner of the FP64 SIMT products (process-wide; off by default).
 * With it on, the first product of each shape with beta = 0 times the tile
 * edges 16, 32 and 64 and keeps the fastest for that shape (the shapes follow
 * D and chi); every tile sums in the same order, so results do not change.
 * Returns the number of shapes tuned so far. */
int tn_set_autotune(int enable);

/* ---- observables (Sec. VI.D; row a14) ----------------------------------- */
typedef struct tn_observables {
    double e_site;    /* -(1/n) sum_links <ZZ> J - h (1/n) sum_t <X>_t */
    double e_link;    /* e_site / 2 */
    double mx[2];     /* <X> per tensor id */
    double mz[2];     /* <Z> per tensor id */
    double zz[4];     /* <Z Z> per link type: (A,h), (B,h), (A,v), (B,v) */
} tn_observables;

/* Observables of the current state from the current environment (which must
 * be the environment of the state's own double layers: call
 * tn_build_double_layer + tn_ctmrg first). */
int tn_measure(void* ctx, tn_observables* obs);

/* ---- 1D iMPS (Sec. III and V: the chain, where the method has an exact answer) ----
 * One-site iMPS A[s][l][r] (d = 2, bond chi, 1 <= chi <= 16) in device memory,
 * transverse-field Ising chain H = -sum Z Z - h sum X.  work: device scratch
 * of at least tn_imps_workspace_bytes(chi) bytes (caller owned, any alignment;
 * the library aligns inside it); stream: cudaStream_t (NULL = legacy default);
 * each call synchronises it.  TN_EINVAL for chi outside 1..16, tau <= 0 or a
 * non-finite h; TN_ENOMEM for a short workspace. */
size_t tn_imps_workspace_bytes(int chi);
/* n_steps plain iTEBD steps with the iMPO (Sec. V.A): A <- Q (g A) P, the
 * optimal truncation through the canonical form of g A (Sec. III), unit norm. */
int tn_imps_itebd(double* dA, int chi, double h, double tau, int n_steps, void* work, size_t bytes, void* stream);
/* One recycling window (Sec. V.B): A_0 = weighted canonical form of A; one
 * plain step gives A~ = Q (g A_0) P; the canonical form of A~ gives its maps;
 * gauge fixing (Sec. III.B.2, started from the polar factor of the kappa = 0
 * block of the leg map Q_c Q) finds U with A~_1 ~ U A_0 U^T (fidelity F,
 * optional out); the
 * renormalised gate G = U^T Q_c Q g P P_c U is applied n_re times to A_0.
 * A is replaced by A_{n_re}. */
int tn_imps_recycle(double* dA, int chi, double h, double tau, int n_re, double* fidelity, void* work,
                    size_t bytes, void* stream);
/* <ZZ>, <X> and the energy per site e = -<ZZ> - h <X> of A (out[0..2], host),
 * from its canonical form. */
int tn_imps_observables(const double* dA, int chi, double h, double* out, void* work, size_t bytes, void* stream);

/* ---- intermediate tensors (for checkpoints and parity checks) ----------- */
#define TN_T_STATE      0   /* A per tensor id: d*D^4 */
#define TN_T_CANON      1   /* weighted canonical tensors A_c (a11): d*D^4 */
#define TN_T_LAMBDA     2   /* canonical weights per link type: D */
#define TN_T_THETA      3   /* Theta = g A_c per tensor id: d*(2D)^4 */
#define TN_T_PRE_P      4   /* pre-truncation P per link type: 2D x D */
#define TN_T_PRE_Q      5   /* pre-truncation Q per link type: D x 2D */
#define TN_T_DOUBLE     6   /* double layer per tensor id: D^8 (a[l][r][d][u]) */
#define TN_T_BOND_ENV   7   /* normalised, PSD bond environment per link type:
                               N4[a][b][a'][b'], (2D)^4 */
#define TN_T_FU_P       8   /* full-update P per link type (balanced) */
#define TN_T_FU_Q       9   /* full-update Q per link type */
#define TN_T_GAUGE_W   10   /* gauge matrices W per link type: D x D */
#define TN_T_GATE_K    11   /* renormalised-gate leg matrices per (tensor, leg l,r,d,u): 2D x D */
#define TN_T_PEPO      12   /* iPEPO g[s'][s][l][r][d][u]: d*d*16 */

/* Copy one intermediate tensor to host; index = tensor id, link type (in the
 * order (A,h), (B,h), (A,v), (B,v); (A,h), (A,v) for the 1-site cell) or
 * tensor*4 + leg.  n must equal the tensor's size (see list above). */
int tn_get_tensor(void* ctx, int which, int index, double* host, size_t n);

/* Projector cutoff (the reading of the cited CTMRG, Sec. VI.B): singular
 * values of the loop matrix below cut * s_1 get a zero inverse square root
 * (the direction is dropped).  Default 1e-12; cut < 0 restores the default.
 * TN_EINVAL for NaN. */
int tn_set_projector_cutoff(void* ctx, double cut);

/* ---- kernel-level entry points (device pointers, used by the parity tests
 *      and usable on their own) ----------------------------------------- */
/* Batched strided C = alpha op(A) op(B) + beta C in double; op = transpose
 * when trans* = 1.  A is m x k (or k x m if transA), row-major with leading
 * dimension lda; likewise B, C; strides in elements between batch entries. */
int tn_gemm_f64(int transA, int transB, int m, int n, int k, double alpha,
                const double* dA, int lda, long long strideA,
                const double* dB, int ldb, long long strideB, double beta,
                double* dC, int ldc, long long strideC, int batch, void* stream);
/* Split-precision C = alpha op(A) op(B) + beta C on the tensor cores
 * (precision TN_TF32X3, TN_BF16X3 or TN_BF16S4; layout and op() as
 * tn_gemm_f64, no batch).  TN_TF32X3 / TN_BF16X3: each FP64 operand is split
 * into head and tail of the tensor-core type, x = hi + lo, and
 * hi.hi + hi.lo + lo.hi is accumulated in FP32 (about 2^-21 relative for
 * TF32, 2^-16 for BF16).  TN_BF16S4: each row of op(A) and column of op(B)
 * is scaled by a power of two and cut (by truncation) into four 8-bit
 * integer slices held exactly in BF16; the ten slice products of the four
 * leading levels are accumulated exactly (integers below 2^24 in FP32,
 * combined in 64-bit integers), so the error is that of the dropped levels,
 * < 20 * 2^-32 (about 2^-27.7) of max|A_i.| max|B_.j| K.  TN_F64S7: the same
 * with seven slices (28 products), error < 2^-51 of max|A_i.| max|B_.j| K,
 * the FP64 rounding level of a K-term sum.  C is written in FP64.
 * This is the contraction arithmetic of the precision form (the paper itself
 * works in double throughout).  d_workspace (device, 256-byte aligned, caller
 * owned) holds the split operands: at least tn_gemm_split_workspace_bytes().
 * Returns TN_ENOMEM if it is smaller, TN_ETIMEOUT if a device-side wait of
 * the kernel expired (C is then invalid); synchronises the stream. */
size_t tn_gemm_split_workspace_bytes(int precision, int m, int n, int k);
int tn_gemm_split(int precision, int transA, int transB, int m, int n, int k, double alpha,
                  const double* dA, int lda, const double* dB, int ldb, double beta,
                  double* dC, int ldc, void* d_workspace, size_t workspace_bytes, void* stream);
/* FP64 throughput probe (no counterpart in the paper): launches, on stream and
 * without synchronising, one kernel in which every thread of 152 x 8 blocks of
 * 256 runs 8 independent fused multiply-add chains of `iters` steps in
 * registers, and returns in *flops the FLOPs it performs (2 per FMA).  Timed
 * with events around the launch it measures the FP64 pipe's peak, the
 * denominator for the FP64 kernels' roofline.  TN_EINVAL for iters < 1. */
int tn_fp64_rate_probe(int iters, double* flops, void* stream);
/* Self-test of the device-side wait limit of the tensor-core kernels (no
 * counterpart in the paper): launches one thread that waits, with the same
 * bounded wait those kernels use, on a barrier nothing ever arrives on.  The
 * wait gives up after about one second, the kernel records the expiry and
 * returns, and the call reports TN_ETIMEOUT (the flag is cleared, the stream
 * and every context stay usable).  Returns TN_OK only if the wait did not
 * expire, which would mean the limit is broken.  Synchronises the stream. */
int tn_selftest_wait_timeout(void* stream);
/* Permute a rank <= 8 tensor: out[i_perm[0]]...[i_perm[r-1]] = in[i_0]..[i_{r-1}],
 * i.e. output axis j is input axis perm[j]; dims are the input dims. */
int tn_permute_f64(const double* d_in, double* d_out, int rank, const int* dims,
                   const int* perm, void* stream);
/* One-sided Jacobi SVD of batch matrices m x n (n <= m <= 112, row-major,
 * consecutive): S descending (batch x n), U (batch x m x n), V (batch x n x n),
 * sign rule: the entry of largest |.| of each column of U is positive. */
int tn_svd_small(const double* dA, int m, int n, int batch, double* dU, double* dS,
                 double* dV, void* stream);
/* Symmetric Jacobi eigendecomposition of batch n x n matrices (n <= 112):
 * eigenvalues ascending (batch x n), eigenvectors as columns of dV. */
int tn_eigh_small(const double* dA, int n, int batch, double* dW, double* dV, void* stream);
/* Top-k singular triplets of one m x m matrix (device), k <= 96: U (m x k),
 * S (k), V (m x k), sign rule applied; warm (optional, m x k) is a starting
 * right basis.  Subspace iteration with Rayleigh-Ritz for m > 112. */
int tn_truncated_svd(void* ctx, const double* dM, int m, int k, double* dU, double* dS,
                     double* dV, const double* warm);

/* Allocation-free variant of tn_truncated_svd (the paper has no counterpart:
 * this is a deployment convenience).  For callers that cannot allocate device
 * memory when they need it -- device memory held by another allocator, code
 * that must not take the device-wide synchronisation of cudaMalloc/cudaFree,
 * or a plugin without a context workspace -- it takes only the caller's
 * buffers (dM: m x m input, dU/dV: m x k, dS: k, warm: optional m x k start)
 * and uses a fixed device array of 2^20 doubles (8 MiB) that the library
 * reserves on every GPU that loads it, until the process exits.
 *  - Limits: k <= 96 and k <= m; the (m, k) scratch need must fit the array
 *    (e.g. m <= 1024 with k <= 64 fits; m <= 112 always fits), otherwise
 *    TN_ESCRATCH and nothing is run.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and caches it for the
 *    process; make that first call before any stream capture begins.  The
 *    cache is not reset-safe: after cudaDeviceReset the cached address is
 *    stale.  Devices with an index of 64 or more are looked up on every call.
 *  - Every call on a device shares the array and leaves its contents behind:
 *    calls that overlap on the GPU (other streams, other threads) race.
 *    Nothing in the array is assumed to start at zero.
 *  - stream: cudaStream_t (NULL = legacy default).  The call waits on the
 *    stream between subspace iterations (it reads convergence data on the
 *    host) and synchronises it before returning.
 *    Returns TN_OK or TN_ENOCONV (subspace iteration cap reached). */
int tn_truncated_svd_noalloc(const double* dM, int m, int k, double* dU, double* dS,
                             double* dV, const double* warm, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TNITE_H */
